// dice.cu -- bulk batched dice (Section 5): Algorithm 3 (per-roll bounds,
// product and threshold formed only on the rare path) and Algorithm 2 (one
// fixed bound, threshold known in advance), as persistent kernels in which
// every warp works alone (no CTA barriers): one thread per batch, one
// Theorem 1 chain per batch attempt.
//
// Rejected batches never serialise anything: attempt a of batch g always
// draws word(seed, g, a) = mix64(seed + G * ((g << 16) | a)), G the golden
// increment.  A thread keeps that counter argument incrementally: +G for the
// next attempt, +G * 2^16 * stride for its next batch.
//  - Fixed bound: a warp fills a tile of batches in shared memory, then
//    writes it back with coalesced 16-byte stores.  By default (sweep form)
//    the tile's attempt-0 words are rolled one batch per lane and the
//    rejected batches swept again from a compacted queue; the older tiled
//    form gives each lane fixed batches that it retries in place.  The batch
//    size k is a template parameter for k <= 8, so the chain is unrolled.
//  - Per-roll bounds: a warp takes groups of 32 consecutive batches.  The
//    fast accept test compares the final word with a float upper bound of the
//    batch product (rounded up at every step), so no exact 64-bit product is
//    formed on the common path.  Batches that fail it are queued (ballot +
//    popc) for the exact test -- exact product, threshold 2^64 mod B --
//    which runs in dense passes of 32; rejected batches go to a retry queue,
//    rerun with the next attempt word, also in dense passes.  Digits go
//    straight to global memory: the lanes of a warp hold consecutive
//    batches, so L2 merges their stores into whole sectors (staging them in
//    shared memory for coalesced stores was measured 22% slower).
#include <algorithm>

#include "brr_common.cuh"
#include "internal.h"
#include "words.cuh"

namespace brr {

constexpr int kDiceBlock = 256;
constexpr int kDiceWarps = kDiceBlock / 32;
constexpr int kFixedTileWords = 768;  // staged digits per warp tile (fixed bound)
constexpr int kMaxRows = 24;          // rows of 32 batches per tile
constexpr int kQueueCap = 64;         // entries per warp queue (per-roll bounds)
constexpr uint64_t kBatchStep = kGolden << 16;  // counter step of one batch

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }

// One die of a fixed bound: b = bm1 + 1, or b = 2^32 (kFull), where the
// digit is the high half of r and the new leftover its low half shifted up.
template <bool kFull>
__device__ __forceinline__ uint32_t fixed_die(uint64_t &r, uint32_t b) {
    if (kFull) {
        const uint32_t a = (uint32_t)(r >> 32);
        r <<= 32;
        return a;
    }
    return chain_step(r, b);
}

// The same at L = 32 (32-bit words): b = 2^32 (kFull) only as a single die,
// whose digit is the whole word.
template <bool kFull>
__device__ __forceinline__ uint32_t fixed_die32(uint32_t &r, uint32_t b) {
    if (kFull) {
        const uint32_t a = r;
        r = 0;
        return a;
    }
    return chain_step32(r, b);
}

// One attempt of a fixed-bound batch: the word of batch g, attempt a from
// source SRC (words.cuh), then K dice (K = 0: kk dice) into dst; returns the
// leftover word, which the caller compares with the threshold.
template <uint32_t SRC, bool kFull, int K>
__device__ __forceinline__ uint64_t fixed_attempt(uint64_t seed, uint64_t g, uint32_t a, uint32_t b,
                                                  uint32_t kk, uint32_t *dst) {
    if constexpr (SRC == BRR_WORDS_SPLITMIX32) {
        uint32_t r = splitmix32_word(seed, g, a);
        if (K) {
#pragma unroll
            for (int i = 0; i < K; i++) dst[i] = fixed_die32<kFull>(r, b);
        } else {
            for (uint32_t i = 0; i < kk; i++) dst[i] = fixed_die32<kFull>(r, b);
        }
        return r;
    } else {
        uint64_t r = SRC == BRR_WORDS_CHACHA20 ? chacha20_word(seed, g, a) : word(seed, g, a);
        if (K) {
#pragma unroll
            for (int i = 0; i < K; i++) dst[i] = fixed_die<kFull>(r, b);
        } else {
            for (uint32_t i = 0; i < kk; i++) dst[i] = fixed_die<kFull>(r, b);
        }
        return r;
    }
}

// ============================================================ fixed bound ==
// Batch g written straight to global memory, retried in place: the tail of
// a run, and the whole run when tiles cannot be used.
template <uint32_t SRC, bool kFull>
__device__ __forceinline__ void fixed_direct_batch(uint64_t g, uint32_t b, uint32_t k,
                                                   uint64_t t_full, uint64_t t_last,
                                                   uint64_t n_rolls, uint64_t seed, uint32_t *out,
                                                   uint32_t max_att, int &e) {
    const uint64_t s = g * k;
    const uint32_t kk = (uint32_t)((n_rolls - s) < k ? (n_rolls - s) : k);
    const uint64_t t = kk == k ? t_full : t_last;
    for (uint32_t att = 0;; att++) {
        if (att >= max_att) { e = BRR_ERETRY; return; }
        if (fixed_attempt<SRC, kFull, 0>(seed, g, att, b, kk, out + s) >= t) return;
    }
}

// K > 0: batches of exactly K dice (unrolled); K == 0: k_rt dice.
template <int K, bool kFull>
__global__ void __launch_bounds__(kDiceBlock)
dice_fixed_kernel(uint32_t b, uint32_t k_rt, uint32_t rows, uint64_t t_full, uint64_t t_last,
                  uint64_t n_rolls, uint64_t seed, uint32_t *__restrict__ out, uint32_t max_att, int *err) {
    __shared__ __align__(16) uint32_t smem[kDiceWarps][kFixedTileWords];
    const uint32_t k = K ? (uint32_t)K : k_rt;
    uint32_t *tile = smem[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const uint64_t n_full = n_rolls / k;  // batches with k dice
    const uint64_t tile_batches = 32ull * rows;
    const uint64_t n_tiles = n_full / tile_batches;
    const uint64_t warp = (uint64_t)blockIdx.x * kDiceWarps + (threadIdx.x >> 5);
    const uint64_t n_warps = (uint64_t)gridDim.x * kDiceWarps;
    int e = 0;

    for (uint64_t t = warp; t < n_tiles; t += n_warps) {
        const uint64_t g0 = t * tile_batches;
        // lane handles batches g0 + 32 v + lane; digits at tile[(32 v + lane) k]
        uint64_t x = seed + kBatchStep * (g0 + lane);  // attempt-0 counter argument
        uint64_t xa = x;
        uint32_t v = 0, att = 0;
        uint32_t *dst = tile + lane * k;
        while (__any_sync(0xffffffffu, v < rows)) {
            if (v < rows) {
                uint64_t r = mix64(xa);
                if (K) {
#pragma unroll
                    for (int i = 0; i < K; i++) dst[i] = fixed_die<kFull>(r, b);
                } else {
                    for (uint32_t i = 0; i < k; i++) dst[i] = fixed_die<kFull>(r, b);
                }
                if (r >= t_full || att + 1 >= max_att) {
                    if (r < t_full) e = BRR_ERETRY;
                    v++;
                    dst += 32 * k;
                    x += kBatchStep * 32;
                    xa = x;
                    att = 0;
                } else {
                    xa += kGolden;
                    att++;
                }
            }
        }
        __syncwarp();
        // coalesced 16-byte stores of the tile
        const uint32_t words = (uint32_t)(tile_batches * k);
        uint4 *dst4 = reinterpret_cast<uint4 *>(out + g0 * k);
        const uint4 *src4 = reinterpret_cast<const uint4 *>(tile);
        for (uint32_t w = lane; w < words / 4; w += 32) dst4[w] = src4[w];
        __syncwarp();
    }

    // tail: batches after the last full tile (including a short last batch),
    // done by the warp that would own the next tile
    if (warp == n_tiles % n_warps) {
        const uint64_t n_batches = (n_rolls + k - 1) / k;
        for (uint64_t g = n_tiles * tile_batches + lane; g < n_batches; g += 32)
            fixed_direct_batch<BRR_WORDS_SPLITMIX64, kFull>(g, b, k, t_full, t_last, n_rolls, seed, out, max_att, e);
    }
    if (e) record_error(err, e);
}

// Sweep form of the fixed-bound kernel (the default): every batch of a warp
// tile first runs its attempt 0, one batch per lane, with no retry logic in
// the loop; the rejected ones are compacted into a queue of tile slots
// (ballot + popc), which is then swept with attempt 1, 2, ... -- the
// survivors of each sweep are written back to the front of the same queue --
// until it is empty.  Then the tile is written back with coalesced 16-byte
// stores.  Lanes never wait on one another's rejections except in the short
// sweeps, and the common path carries no per-lane bookkeeping.
template <int K>
struct SweepShape {
    static constexpr uint32_t TB = 32u * (1024u / (32u * K));  // batches per tile
    static constexpr uint32_t TW = TB * K;                     // words per tile
};

template <int K, bool kFull, uint32_t SRC>
__global__ void __launch_bounds__(kDiceBlock)
dice_fixed_sweep_kernel(uint32_t b, uint64_t t_full, uint64_t t_last, uint64_t n_rolls, uint64_t seed,
                        uint32_t *__restrict__ out, uint32_t max_att, int *err) {
    constexpr uint32_t TB = SweepShape<K>::TB, TW = SweepShape<K>::TW;
    __shared__ __align__(16) uint32_t smem_tile[kDiceWarps][TW];
    __shared__ uint16_t smem_q[kDiceWarps][TB];
    uint32_t *tile = smem_tile[threadIdx.x >> 5];
    uint16_t *q = smem_q[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const uint64_t n_full = n_rolls / K;  // batches with K dice
    const uint64_t n_tiles = n_full / TB;
    const uint64_t warp = (uint64_t)blockIdx.x * kDiceWarps + (threadIdx.x >> 5);
    const uint64_t n_warps = (uint64_t)gridDim.x * kDiceWarps;
    int e = 0;

    for (uint64_t t = warp; t < n_tiles; t += n_warps) {
        const uint64_t g0 = t * TB;
        // attempt 0 of every batch of the tile
        uint64_t x = seed + kBatchStep * (g0 + lane);
        int rq = 0;
#pragma unroll 4
        for (uint32_t slot = lane; slot < TB; slot += 32, x += kBatchStep * 32) {
            uint32_t *p = tile + slot * K;
            uint64_t left;
            if constexpr (SRC == BRR_WORDS_SPLITMIX64) {
                // the SplitMix64 counter argument is carried from batch to batch
                uint64_t r = mix64(x);
#pragma unroll
                for (int i = 0; i < K; i++) p[i] = fixed_die<kFull>(r, b);
                left = r;
            } else {
                left = fixed_attempt<SRC, kFull, K>(seed, g0 + slot, 0, b, K, p);
            }
            const bool rej = left < t_full;
            const uint32_t m = __ballot_sync(0xffffffffu, rej);
            if (rej) q[rq + __popc(m & lanemask_lt())] = (uint16_t)slot;
            rq += __popc(m);
        }
        // sweeps of the rejected batches, attempt a = 1, 2, ...
        for (uint32_t a = 1; rq > 0; a++) {
            __syncwarp();
            if (a >= max_att) {
                e = BRR_ERETRY;
                break;
            }
            const int n = rq;
            rq = 0;
            for (int c = 0; c < n; c += 32) {
                const bool has = c + (int)lane < n;
                const uint32_t slot = has ? q[c + lane] : 0;
                __syncwarp();  // every lane has read its entry before any is overwritten
                bool rej = false;
                if (has) rej = fixed_attempt<SRC, kFull, K>(seed, g0 + slot, a, b, K, tile + slot * K) < t_full;
                // survivors go to the front: at most c + 32 entries so far
                const uint32_t m = __ballot_sync(0xffffffffu, rej);
                if (rej) q[rq + __popc(m & lanemask_lt())] = (uint16_t)slot;
                rq += __popc(m);
            }
        }
        __syncwarp();
        const uint4 *src4 = reinterpret_cast<const uint4 *>(tile);
        uint4 *dst4 = reinterpret_cast<uint4 *>(out + g0 * K);
#pragma unroll 4
        for (uint32_t w = lane; w < TW / 4; w += 32) dst4[w] = src4[w];
        __syncwarp();
    }

    // tail: batches after the last full tile (including a short last batch),
    // done by the warp that would own the next tile
    if (warp == n_tiles % n_warps) {
        const uint64_t n_batches = (n_rolls + K - 1) / K;
        for (uint64_t g = n_tiles * TB + lane; g < n_batches; g += 32)
            fixed_direct_batch<SRC, kFull>(g, b, K, t_full, t_last, n_rolls, seed, out, max_att, e);
    }
    if (e) record_error(err, e);
}

// Untiled form for batch sizes whose tiles would not fit or unaligned
// outputs: one thread per batch, grid-stride.
template <uint32_t SRC, bool kFull>
__global__ void __launch_bounds__(kDiceBlock)
dice_fixed_direct_kernel(uint32_t b, uint32_t k, uint64_t t_full, uint64_t t_last,
                         uint64_t n_rolls, uint64_t seed, uint32_t *__restrict__ out, uint32_t max_att, int *err) {
    const uint64_t n_batches = (n_rolls + k - 1) / k;
    int e = 0;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_batches;
         g += (uint64_t)gridDim.x * blockDim.x)
        fixed_direct_batch<SRC, kFull>(g, b, k, t_full, t_last, n_rolls, seed, out, max_att, e);
    if (e) record_error(err, e);
}

// ========================================================= per-roll bounds ==
struct VarWarp {
    uint64_t er[kQueueCap];   // exact-test queue: final word of the attempt
    uint32_t eg[kQueueCap];   //                   batch
    uint32_t rg[kQueueCap];   // retry queue:      batch
    uint32_t ra[kQueueCap];   //                   attempt to run next
};

// Float upper bound of b = bm1 + 1 (rounded up), for the running product.
__device__ __forceinline__ float bound_up(uint32_t bm1) {
    return __fadd_ru(__uint2float_ru(bm1), 1.0f);
}

// Word, die and fast test of the per-roll-bound kernel for a word source:
// SplitMix64 or ChaCha20 words at L = 64, or the 32-bit source at L = 32
// (the word in the low half of r).
template <uint32_t SRC>
__device__ __forceinline__ uint64_t var_word(uint64_t seed, uint64_t g, uint32_t a) {
    if constexpr (SRC == BRR_WORDS_CHACHA20) return chacha20_word(seed, g, a);
    else if constexpr (SRC == BRR_WORDS_SPLITMIX32) return splitmix32_word(seed, g, a);
    else return word(seed, g, a);
}

// One Theorem 1 step for a bound given as bm1 = b - 1; at L = 32 the product
// r * b = r * bm1 + r is below 2^64 for every b <= 2^32.
template <uint32_t SRC>
__device__ __forceinline__ uint32_t var_die(uint64_t &r, uint32_t bm1) {
    if constexpr (SRC == BRR_WORDS_SPLITMIX32) {
        const uint32_t r32 = (uint32_t)r;
        const uint64_t p = (uint64_t)r32 * bm1 + r32;
        r = (uint32_t)p;
        return (uint32_t)(p >> 32);
    } else {
        return chain_step_m1(r, bm1);
    }
}

// r >= bf, with bf >= B the rounded-up float product: accept at once.
template <uint32_t SRC>
__device__ __forceinline__ bool var_fast(uint64_t r, float bf) {
    if constexpr (SRC == BRR_WORDS_SPLITMIX32) return __uint2float_rd((uint32_t)r) >= bf;
    else return __ull2float_rd(r) >= bf;
}

// Exact test of a finished attempt with final word r (Algorithm 3): the
// product B of the batch's bounds (kept as B - 1, exact) and r >= 2^L mod B.
// Clears `valid` if the product exceeds 2^L.
template <uint32_t SRC>
__device__ __forceinline__ bool exact_accept(const uint32_t *__restrict__ bm1, uint32_t s,
                                             uint32_t e, uint64_t r, bool &valid) {
    uint64_t Bm1 = 0;
    bool ok = true;
    for (uint32_t x = s; x < e; x++) ok = prod_m1_step(Bm1, __ldg(&bm1[x])) && ok;
    if constexpr (SRC == BRR_WORDS_SPLITMIX32) {
        valid = ok && Bm1 <= 0xFFFFFFFFull;
        if (Bm1 >= 0xFFFFFFFFull) return true;  // B = 2^32: threshold 0 (or invalid)
        const uint32_t B = (uint32_t)Bm1 + 1u;
        return (uint32_t)r >= (0u - B) % B;
    } else {
        valid = ok;
        return r > Bm1 || r >= threshold_from_m1(Bm1);
    }
}

// Appends (a, b) for every lane with flag set to a warp queue of length q.
template <typename A, typename B>
__device__ __forceinline__ void queue_push(bool flag, A a, B b, A *qa, B *qb, int &q) {
    const uint32_t m = __ballot_sync(0xffffffffu, flag);
    if (flag) {
        const int pos = q + __popc(m & lanemask_lt());
        qa[pos] = a;
        qb[pos] = b;
    }
    q += __popc(m);
    __syncwarp();
}

template <bool kImplicit>
__device__ __forceinline__ void batch_range(const uint32_t *off, uint32_t g, uint32_t &s, uint32_t &e) {
    if (kImplicit) {
        s = g;
        e = g + 1;
    } else {
        s = __ldg(&off[g]);
        e = __ldg(&off[g + 1]);
    }
}

// Dense pass over up to 32 queued exact tests; rejected batches go to the
// retry queue with attempt 1.
template <bool kImplicit, uint32_t SRC>
__device__ void exact_pass(VarWarp &W, int &eq, int &rq, const uint32_t *bm1, const uint32_t *off,
                           int &err) {
    const uint32_t lane = lane_id();
    const int take = eq < 32 ? eq : 32;
    const int base = eq - take;
    const bool has = (int)lane < take;
    uint32_t g = 0;
    uint64_t r = 0;
    if (has) {
        g = W.eg[base + lane];
        r = W.er[base + lane];
    }
    __syncwarp();
    eq = base;
    bool rej = false;
    if (has) {
        uint32_t s, e;
        batch_range<kImplicit>(off, g, s, e);
        bool valid;
        rej = !exact_accept<SRC>(bm1, s, e, r, valid);
        if (!valid) {
            err = BRR_EINVAL;
            rej = false;
        }
    }
    queue_push<uint32_t, uint32_t>(rej, g, 1u, W.rg, W.ra, rq);
}

// Dense pass over up to 32 queued retries: the next attempt word, digits
// straight to global memory over the rejected attempt's, exact test inline;
// rejected again -> queued with the following attempt.
template <bool kImplicit, uint32_t SRC>
__device__ void retry_pass(VarWarp &W, int &rq, const uint32_t *bm1, const uint32_t *off,
                           uint64_t seed, uint32_t *out, uint32_t max_att, int &err) {
    const uint32_t lane = lane_id();
    const int take = rq < 32 ? rq : 32;
    const int base = rq - take;
    const bool has = (int)lane < take;
    uint32_t g = 0, att = 0;
    if (has) {
        g = W.rg[base + lane];
        att = W.ra[base + lane];
    }
    __syncwarp();
    rq = base;
    bool rej = false;
    if (has) {
        if (att >= max_att) {
            err = BRR_ERETRY;
        } else {
            uint32_t s, e;
            batch_range<kImplicit>(off, g, s, e);
            uint64_t r = var_word<SRC>(seed, g, att);
            for (uint32_t x = s; x < e; x++) out[x] = var_die<SRC>(r, __ldg(&bm1[x]));
            bool valid;
            rej = !exact_accept<SRC>(bm1, s, e, r, valid);
        }
    }
    queue_push<uint32_t, uint32_t>(rej, g, att + 1, W.rg, W.ra, rq);
}

// The per-roll-bound kernel of the 32-bit word source (L = 32): batches of
// product at most 2^32, queued exact tests and retries that re-read their
// offsets and bounds.  kImplicit: batch g is roll g (off unused).
template <bool kImplicit, uint32_t SRC>
__global__ void __launch_bounds__(kDiceBlock, 8)
dice_var_l32_kernel(const uint32_t *__restrict__ bm1, const uint32_t *__restrict__ off,
                    uint32_t n_batches, uint32_t n_rolls, uint64_t seed, uint32_t *__restrict__ out,
                    uint32_t max_att, int *err) {
    __shared__ VarWarp smem[kDiceWarps];
    VarWarp &W = smem[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const uint32_t warp = blockIdx.x * kDiceWarps + (threadIdx.x >> 5);
    const uint32_t n_warps = gridDim.x * kDiceWarps;
    const uint32_t n_groups = (uint32_t)(((uint64_t)n_batches + 31) / 32);
    int eq = 0, rq = 0, e = 0;
    // attempt-0 counter argument of this lane's batch, advanced per group
    uint64_t xc = seed + kBatchStep * ((uint64_t)warp * 32 + lane);
    const uint64_t xstep = kBatchStep * 32 * (uint64_t)n_warps;

    for (uint32_t grp = warp; grp < n_groups; grp += n_warps, xc += xstep) {
        const uint32_t g0 = grp * 32;
        const uint32_t nb = min(32u, n_batches - g0);
        const uint32_t g = g0 + lane;
        const bool active = lane < nb;
        uint32_t s, en;
        bool bad = false;
        if (kImplicit) {
            s = g;
            en = g + 1;
        } else {
            const uint32_t mine = active ? __ldg(&off[g]) : 0;
            const uint32_t R1 = __ldg(&off[g0 + nb]);
            const uint32_t next = __shfl_down_sync(0xffffffffu, mine, 1);
            s = mine;
            en = lane + 1 == nb ? R1 : next;
            bad = active && (en < s || en > n_rolls);
            if (lane == 0 && grp == 0 && mine != 0) bad = true;
            if (lane == 0 && g0 + nb == n_batches && R1 != n_rolls) bad = true;
        }
        if (__any_sync(0xffffffffu, bad)) {
            e = BRR_EINVAL;
            continue;
        }
        bool fast = true;
        uint64_t r = 0;
        if (active) {
            r = SRC == BRR_WORDS_SPLITMIX64 ? mix64(xc) : var_word<SRC>(seed, g, 0);
            float bf = 1.0f;
            // a batch holds k = en - s dice; the first six are unrolled, with
            // loads and stores at constant offsets from per-lane bases.  The
            // digits go straight to global memory: a warp's lanes write
            // consecutive batches, so L2 merges them into whole sectors
            // (measured faster than staging them in shared memory).
            const uint32_t k = en - s;
            const uint32_t *src = bm1 + s;
            uint32_t *dst = out + s;
#pragma unroll
            for (uint32_t i = 0; i < 6; i++) {
                if (i < k) {
                    const uint32_t m1 = __ldg(src + i);
                    dst[i] = var_die<SRC>(r, m1);
                    bf = __fmul_ru(bf, bound_up(m1));
                }
            }
            for (uint32_t i = 6; i < k; i++) {
                const uint32_t m1 = __ldg(src + i);
                dst[i] = var_die<SRC>(r, m1);
                bf = __fmul_ru(bf, bound_up(m1));
            }
            // r >= bf >= B implies r >= B > threshold: accept without the
            // exact product (r < 2^64, so this also certifies B <= 2^64)
            fast = var_fast<SRC>(r, bf);
        }
        queue_push<uint64_t, uint32_t>(!fast, r, g, W.er, W.eg, eq);
        while (eq >= 32) exact_pass<kImplicit, SRC>(W, eq, rq, bm1, off, e);
        while (rq >= 32) retry_pass<kImplicit, SRC>(W, rq, bm1, off, seed, out, max_att, e);
    }
    while (eq > 0) exact_pass<kImplicit, SRC>(W, eq, rq, bm1, off, e);
    while (rq > 0) retry_pass<kImplicit, SRC>(W, rq, bm1, off, seed, out, max_att, e);
    if (e) record_error(err, e);
}

// ------------------------------------------- per-roll bounds at L = 64 --
// The kernel the SplitMix64 and ChaCha20 word sources use.  Per group of 32
// batches (one per lane):
//  - the six first dice of every batch are always rolled: a die past the
//    batch's end gets bound 1 (bm1 = 0), which leaves the leftover word and
//    the product bound unchanged and gives digit 0, and its load and store
//    are predicated off.  The loop has no branches, so the leftover word's
//    registers need no copies at merge points; batches of more than six
//    dice (none in the bulk workload) continue in a loop of their own.
//  - the word, its counter and the leftover are 32-bit halves
//    (mix64_halves, chain_step_m1_halves): no 64-bit register pairs.
//  - a batch that fails the fast test is queued for the exact test with its
//    word and its bounds, which it carries in the warp's shared-memory queue:
//    the exact-test and retry passes read no global memory except the
//    bounds of batches longer than six dice.  (Re-reading offsets and bounds
//    there was measured as a quarter of the kernel's time.)
constexpr int kPendCap = 64;    // pending batches per warp
constexpr int kPendDice = 6;    // bounds carried per pending batch

struct PendWarp {
    uint32_t rl[kPendCap], rh[kPendCap];  // leftover of attempt 0 (tested exactly first)
    uint32_t g[kPendCap], s[kPendCap];    // batch and its first roll
    uint32_t k[kPendCap], a[kPendCap];    // dice, and the attempt to run next
    uint32_t b[kPendDice][kPendCap];      // bm1 of the batch's first dice
};

// bf <- bf * (bm1 + 1), one rounding up: bf * m + bf with m >= bm1.
__device__ __forceinline__ float bound_mul_up(float bf, uint32_t bm1) {
    return __fmaf_ru(bf, __uint2float_ru(bm1), bf);
}

// Exact test of a finished attempt: the batch product B (kept as B - 1) and
// r >= 2^64 mod B; bounds from registers (k <= kPendDice) or global memory.
// Clears `valid` when the product exceeds 2^64.
__device__ __forceinline__ bool exact_accept_pend(const uint32_t *m, uint32_t k, const uint32_t *gsrc,
                                                  uint32_t rl, uint32_t rh, bool &valid) {
    uint64_t Bm1 = 0;
    bool ok = true;
    if (k <= kPendDice) {
#pragma unroll
        for (uint32_t i = 0; i < kPendDice; i++)
            if (i < k) ok = prod_m1_step(Bm1, m[i]) && ok;
    } else {
        for (uint32_t i = 0; i < k; i++) ok = prod_m1_step(Bm1, __ldg(gsrc + i)) && ok;
    }
    valid = ok;
    const uint64_t r = ((uint64_t)rh << 32) | rl;
    return r > Bm1 || r >= threshold_from_m1(Bm1);
}

// Fast test of a batch of at most kPendDice dice with float product bound
// bf >= B (two upward roundings per die, so bf <= B (1 + 2^-23)^12 <
// B (1 + 2^-19.4)) and leftover high word rh: accept when r >= T for an
// upper bound T of Lemire's threshold t = 2^64 mod B = 2^64 - qB,
// q = floor(2^64 / B):
//  - q' = floor(rcp(bf) 2^64 (1 - 2^-21)), the reciprocal within one ulp and
//    every rounding downward, so q' <= 2^64 / bf <= 2^64 / B, hence q' <= q;
//  - B' = bf (1 - 2^-19) rounded down < B;
//  - T = 2^64 - q' B' rounded up >= 2^64 - qB = t.
// r >= rh 2^32 >= T >= t then accepts without the exact product.  T exceeds
// t by q B - q' B', a sliver unless q' < q, so only the batches the exact
// test rejects (3.5% of the bulk workload) and a few near those go to the
// exact test, against 8.2% with the plain test r >= bf.  A product above
// 2^64 (invalid) gives q' = 0 and T = 2^64 (or a NaN once bf overflows):
// never accepted here, so the exact test reports it.
__device__ __forceinline__ bool fast_accept(float bf, uint32_t rh) {
    const float blo = __fmul_rd(bf, 1.0f - 0x1p-19f);
    float rc;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rc) : "f"(bf));
    const float q = floorf(__fmul_rd(rc, 0x1p64f * (1.0f - 0x1p-21f)));
    const float T = __fmaf_ru(-q, blo, 0x1p64f);
    return __uint2float_rd(rh) >= T * 0x1p-32f;
}

template <uint32_t SRC>
__device__ __forceinline__ void word_halves(uint64_t seed, uint64_t g, uint32_t a, uint32_t &rl, uint32_t &rh) {
    const uint64_t w = SRC == BRR_WORDS_CHACHA20 ? chacha20_word(seed, g, a) : word(seed, g, a);
    rl = (uint32_t)w;
    rh = (uint32_t)(w >> 32);
}

// One dense pass over up to 32 pending batches (the last ones queued).
// Attempt 0 is tested exactly with its stored leftover; a later attempt
// draws its word, rolls its dice over the rejected attempt's digits and is
// tested exactly.  Rejected batches are queued again with the next attempt.
template <uint32_t SRC>
__device__ void pending_pass(PendWarp &W, int &pq, const uint32_t *bm1, uint64_t seed, uint32_t *out,
                             uint32_t max_att, int &err) {
    const uint32_t lane = lane_id();
    const int take = pq < 32 ? pq : 32;
    const int base = pq - take;
    const bool has = (int)lane < take;
    uint32_t g = 0, s = 0, k = 0, att = 0, rl = 0, rh = 0, m[kPendDice];
#pragma unroll
    for (int i = 0; i < kPendDice; i++) m[i] = 0;
    if (has) {
        const int x = base + lane;
        g = W.g[x];
        s = W.s[x];
        k = W.k[x];
        att = W.a[x];
        rl = W.rl[x];
        rh = W.rh[x];
#pragma unroll
        for (int i = 0; i < kPendDice; i++) m[i] = W.b[i][x];
    }
    __syncwarp();
    pq = base;
    bool rej = false;
    if (has) {
        if (att >= max_att) {
            err = BRR_ERETRY;
        } else {
            if (att > 0) {
                word_halves<SRC>(seed, g, att, rl, rh);
                uint32_t *dst = out + s;
                if (k <= kPendDice) {
#pragma unroll
                    for (uint32_t i = 0; i < kPendDice; i++) {
                        const uint32_t d = chain_step_m1_halves(rl, rh, m[i]);
                        if (i < k) dst[i] = d;
                    }
                } else {
                    for (uint32_t i = 0; i < k; i++) dst[i] = chain_step_m1_halves(rl, rh, __ldg(bm1 + s + i));
                }
            }
            bool valid;
            rej = !exact_accept_pend(m, k, bm1 + s, rl, rh, valid);
            if (!valid) {
                err = BRR_EINVAL;
                rej = false;
            }
        }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, rej);
    if (rej) {
        const int x = pq + __popc(bal & lanemask_lt());
        W.g[x] = g;
        W.s[x] = s;
        W.k[x] = k;
        W.a[x] = att + 1;
#pragma unroll
        for (int i = 0; i < kPendDice; i++) W.b[i][x] = m[i];
    }
    pq += __popc(bal);
    __syncwarp();
}

// kImplicit: batch g is roll g (the unbatched form; off unused).  SRC:
// BRR_WORDS_SPLITMIX64 (the counter argument kept incrementally) or
// BRR_WORDS_CHACHA20 (more registers: fewer blocks per SM).
template <bool kImplicit, uint32_t SRC>
__global__ void __launch_bounds__(kDiceBlock, SRC == BRR_WORDS_CHACHA20 ? 4 : 6)
dice_var_kernel(const uint32_t *__restrict__ bm1, const uint32_t *__restrict__ off, uint32_t n_batches,
                uint32_t n_rolls, uint64_t seed, uint32_t *__restrict__ out, uint32_t max_att, int *err) {
    __shared__ PendWarp smem[kDiceWarps];
    PendWarp &W = smem[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const uint32_t warp = blockIdx.x * kDiceWarps + (threadIdx.x >> 5);
    const uint32_t n_warps = gridDim.x * kDiceWarps;
    const uint32_t n_groups = (uint32_t)(((uint64_t)n_batches + 31) / 32);
    int pq = 0, e = 0;
    // attempt-0 counter argument of this lane's batch, advanced per group
    const uint64_t x0 = seed + kBatchStep * ((uint64_t)warp * 32 + lane);
    uint32_t xl = (uint32_t)x0, xh = (uint32_t)(x0 >> 32);
    const uint64_t xs = kBatchStep * 32 * (uint64_t)n_warps;
    const uint32_t xsl = (uint32_t)xs, xsh = (uint32_t)(xs >> 32);

    for (uint32_t grp = warp; grp < n_groups; grp += n_warps) {
        const uint32_t g0 = grp * 32;
        const uint32_t nb = min(32u, n_batches - g0);
        const uint32_t g = g0 + lane;
        const bool active = lane < nb;
        uint32_t s, en;
        bool bad = false;
        if (kImplicit) {
            s = g;
            en = active ? g + 1 : g;
        } else {
            const uint32_t mine = active ? __ldg(&off[g]) : 0;
            const uint32_t R1 = __ldg(&off[g0 + nb]);
            const uint32_t next = __shfl_down_sync(0xffffffffu, mine, 1);
            s = mine;
            en = lane + 1 == nb ? R1 : (active ? next : mine);
            bad = active && (en < s || en > n_rolls);
            if (lane == 0 && grp == 0 && mine != 0) bad = true;
            if (lane == 0 && g0 + nb == n_batches && R1 != n_rolls) bad = true;
        }
        uint32_t rl, rh;
        if (SRC == BRR_WORDS_SPLITMIX64) mix64_halves(xl, xh, rl, rh);
        add64_halves(xl, xh, xsl, xsh);
        if (__any_sync(0xffffffffu, bad)) {
            e = BRR_EINVAL;
            continue;
        }
        const uint32_t k = en - s;  // 0 on inactive lanes
        const uint32_t *src = bm1 + s;
        uint32_t *dst = out + s;
        uint32_t m[kPendDice];
#pragma unroll
        for (uint32_t i = 0; i < kPendDice; i++) m[i] = i < k ? __ldg(src + i) : 0u;
        if (SRC == BRR_WORDS_CHACHA20) word_halves<SRC>(seed, g, 0, rl, rh);
        float bf = 1.0f;
#pragma unroll
        for (uint32_t i = 0; i < kPendDice; i++) {
            const uint32_t d = chain_step_m1_halves(rl, rh, m[i]);
            bf = bound_mul_up(bf, m[i]);
            if (i < k) dst[i] = d;
        }
        if (__any_sync(0xffffffffu, k > kPendDice)) {
            for (uint32_t i = kPendDice; i < k; i++) {
                const uint32_t m1 = __ldg(src + i);
                dst[i] = chain_step_m1_halves(rl, rh, m1);
                bf = bound_mul_up(bf, m1);
            }
        }
        // more than kPendDice dice: bf may exceed B by more than T allows for;
        // there r >= rh 2^32 >= bf >= B > t (which also certifies B <= 2^64)
        const bool fast = !active || (k <= kPendDice ? fast_accept(bf, rh) : __uint2float_rd(rh) >= bf * 0x1p-32f);
        const uint32_t bal = __ballot_sync(0xffffffffu, !fast);
        if (!fast) {
            const int x = pq + __popc(bal & lanemask_lt());
            W.rl[x] = rl;
            W.rh[x] = rh;
            W.g[x] = g;
            W.s[x] = s;
            W.k[x] = k;
            W.a[x] = 0;
#pragma unroll
            for (int i = 0; i < kPendDice; i++) W.b[i][x] = m[i];
        }
        pq += __popc(bal);
        __syncwarp();
        while (pq >= 32) pending_pass<SRC>(W, pq, bm1, seed, out, max_att, e);
    }
    while (pq > 0) pending_pass<SRC>(W, pq, bm1, seed, out, max_att, e);
    if (e) record_error(err, e);
}

// ============================================================ self-test ==
__global__ void threshold_test_kernel(const uint64_t *B, uint64_t *t, uint64_t n) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = B[x];
        t[x] = b == 0 ? 0 : lemire_threshold(b);
    }
}

brr_status launch_threshold_test(const uint64_t *B, uint64_t *t, uint64_t n, cudaStream_t stream) {
    if (n == 0) return BRR_OK;
    const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, 4096);
    threshold_test_kernel<<<grid, 256, 0, stream>>>(B, t, n);
    return cuda_status(cudaGetLastError());
}

// ============================================================== launchers ==
template <typename Kern>
static int persistent_grid(brr_ctx *ctx, Kern kernel, uint64_t blocks_needed) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kDiceBlock, 0);
    if (per_sm < 1) per_sm = 1;
    const uint64_t full = (uint64_t)per_sm * (uint64_t)ctx->num_sms;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(full, blocks_needed));
}

template <bool kImplicit, uint32_t SRC>
static void launch_dice_var_one(brr_ctx *ctx, const uint32_t *bm1, const uint32_t *off, uint64_t n_batches,
                                uint64_t n_rolls, uint64_t seed, uint32_t *out, cudaStream_t stream) {
    const uint64_t groups = (n_batches + 31) / 32;
    const uint64_t blocks_needed = (groups + kDiceWarps - 1) / kDiceWarps;
    const uint32_t max_att = ctx->attempt_limit;
    if constexpr (SRC == BRR_WORDS_SPLITMIX32) {
        const int grid = persistent_grid(ctx, dice_var_l32_kernel<kImplicit, SRC>, blocks_needed);
        dice_var_l32_kernel<kImplicit, SRC><<<grid, kDiceBlock, 0, stream>>>(
            bm1, off, (uint32_t)n_batches, (uint32_t)n_rolls, seed, out, max_att, ctx->d_err);
    } else {
        const int grid = persistent_grid(ctx, dice_var_kernel<kImplicit, SRC>, blocks_needed);
        dice_var_kernel<kImplicit, SRC><<<grid, kDiceBlock, 0, stream>>>(
            bm1, off, (uint32_t)n_batches, (uint32_t)n_rolls, seed, out, max_att, ctx->d_err);
    }
}

template <uint32_t SRC>
static void launch_dice_var_src(brr_ctx *ctx, const uint32_t *bm1, const uint32_t *off, uint64_t n_batches,
                                uint64_t n_rolls, uint64_t seed, uint32_t *out, cudaStream_t stream) {
    if (off == nullptr) launch_dice_var_one<true, SRC>(ctx, bm1, off, n_batches, n_rolls, seed, out, stream);
    else launch_dice_var_one<false, SRC>(ctx, bm1, off, n_batches, n_rolls, seed, out, stream);
}

brr_status launch_dice_var(brr_ctx *ctx, const uint32_t *bm1, const uint32_t *off,
                           uint64_t n_batches, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                           cudaStream_t stream, uint32_t source) {
    if (n_batches == 0) return BRR_OK;
    if (source == BRR_WORDS_CHACHA20)
        launch_dice_var_src<BRR_WORDS_CHACHA20>(ctx, bm1, off, n_batches, n_rolls, seed, out, stream);
    else if (source == BRR_WORDS_SPLITMIX32)
        launch_dice_var_src<BRR_WORDS_SPLITMIX32>(ctx, bm1, off, n_batches, n_rolls, seed, out, stream);
    else
        launch_dice_var_src<BRR_WORDS_SPLITMIX64>(ctx, bm1, off, n_batches, n_rolls, seed, out, stream);
    return cuda_status(cudaGetLastError());
}

template <int K, bool kFull>
static void launch_fixed_tiles(brr_ctx *ctx, uint32_t b, uint32_t k, uint32_t rows, uint64_t t_full,
                               uint64_t t_last, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                               cudaStream_t stream) {
    const uint64_t tiles = (n_rolls / k) / (32ull * rows);
    const uint64_t blocks_needed = std::max<uint64_t>(1, (tiles + kDiceWarps - 1) / kDiceWarps);
    const int grid = persistent_grid(ctx, dice_fixed_kernel<K, kFull>, blocks_needed);
    dice_fixed_kernel<K, kFull><<<grid, kDiceBlock, 0, stream>>>(b, k, rows, t_full, t_last, n_rolls,
                                                                 seed, out, ctx->attempt_limit, ctx->d_err);
}

template <int K, bool kFull, uint32_t SRC = BRR_WORDS_SPLITMIX64>
static void launch_fixed_sweep(brr_ctx *ctx, uint32_t b, uint64_t t_full, uint64_t t_last, uint64_t n_rolls,
                               uint64_t seed, uint32_t *out, cudaStream_t stream) {
    const uint64_t tiles = (n_rolls / K) / SweepShape<K>::TB;
    const uint64_t blocks_needed = std::max<uint64_t>(1, (tiles + kDiceWarps - 1) / kDiceWarps);
    const int grid = persistent_grid(ctx, dice_fixed_sweep_kernel<K, kFull, SRC>, blocks_needed);
    dice_fixed_sweep_kernel<K, kFull, SRC><<<grid, kDiceBlock, 0, stream>>>(b, t_full, t_last, n_rolls, seed,
                                                                            out, ctx->attempt_limit, ctx->d_err);
}

template <uint32_t SRC, bool kFull>
static void launch_fixed_direct(brr_ctx *ctx, uint32_t b, uint32_t k, uint64_t t_full, uint64_t t_last,
                                uint64_t n_rolls, uint64_t seed, uint32_t *out, cudaStream_t stream) {
    const uint64_t n_batches = (n_rolls + k - 1) / k;
    const uint64_t blocks = (n_batches + kDiceBlock - 1) / kDiceBlock;
    const int grid = persistent_grid(ctx, dice_fixed_direct_kernel<SRC, kFull>, blocks);
    dice_fixed_direct_kernel<SRC, kFull><<<grid, kDiceBlock, 0, stream>>>(b, k, t_full, t_last, n_rolls, seed,
                                                                          out, ctx->attempt_limit, ctx->d_err);
}

template <bool kFull>
static void dispatch_fixed(brr_ctx *ctx, uint32_t b, uint32_t k, uint32_t rows, uint64_t t_full,
                           uint64_t t_last, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                           cudaStream_t stream) {
    if (ctx->tune.fixed_sweep) {
#define BRR_SWEEP_CASE(KK) \
    case KK: launch_fixed_sweep<KK, kFull>(ctx, b, t_full, t_last, n_rolls, seed, out, stream); return;
        switch (k) {
            BRR_SWEEP_CASE(1) BRR_SWEEP_CASE(2) BRR_SWEEP_CASE(3) BRR_SWEEP_CASE(4)
            BRR_SWEEP_CASE(5) BRR_SWEEP_CASE(6) BRR_SWEEP_CASE(7) BRR_SWEEP_CASE(8)
            default: break;
        }
#undef BRR_SWEEP_CASE
    }
#define BRR_FIXED_CASE(KK) \
    case KK: launch_fixed_tiles<KK, kFull>(ctx, b, k, rows, t_full, t_last, n_rolls, seed, out, stream); break;
    switch (k) {
        BRR_FIXED_CASE(1) BRR_FIXED_CASE(2) BRR_FIXED_CASE(3) BRR_FIXED_CASE(4)
        BRR_FIXED_CASE(5) BRR_FIXED_CASE(6) BRR_FIXED_CASE(7) BRR_FIXED_CASE(8)
        default: launch_fixed_tiles<0, kFull>(ctx, b, k, rows, t_full, t_last, n_rolls, seed, out, stream);
    }
#undef BRR_FIXED_CASE
}

brr_status launch_dice_fixed(brr_ctx *ctx, uint32_t bm1, uint32_t k, uint64_t t_full,
                             uint64_t t_last, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                             cudaStream_t stream) {
    if (n_rolls == 0) return BRR_OK;
    const bool full = bm1 == 0xFFFFFFFFu;
    const uint32_t b = bm1 + 1;  // unused (wraps to 0) when full
    // rows of 32 batches per warp tile; tiles start 16-byte aligned in out
    // (32 * rows * k words), so out itself must be 16-byte aligned
    const uint32_t rows = std::min<uint32_t>(kMaxRows, kFixedTileWords / (32 * k));
    const bool aligned = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    if (rows == 0 || !aligned) {
        if (full) launch_fixed_direct<BRR_WORDS_SPLITMIX64, true>(ctx, b, k, t_full, t_last, n_rolls, seed, out, stream);
        else launch_fixed_direct<BRR_WORDS_SPLITMIX64, false>(ctx, b, k, t_full, t_last, n_rolls, seed, out, stream);
        return cuda_status(cudaGetLastError());
    }
    if (full) dispatch_fixed<true>(ctx, b, k, rows, t_full, t_last, n_rolls, seed, out, stream);
    else dispatch_fixed<false>(ctx, b, k, rows, t_full, t_last, n_rolls, seed, out, stream);
    return cuda_status(cudaGetLastError());
}

// Fixed-bound dice on the ChaCha20 or 32-bit source: the sweep kernel for
// 1 <= k <= 8 into a 16-byte-aligned output, else (and for b = 2^32) one
// thread per batch.
template <uint32_t SRC>
static void dispatch_fixed_src(brr_ctx *ctx, uint32_t b, uint32_t k, bool full, bool aligned, uint64_t t_full,
                               uint64_t t_last, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                               cudaStream_t stream) {
    if (full) {
        launch_fixed_direct<SRC, true>(ctx, b, k, t_full, t_last, n_rolls, seed, out, stream);
        return;
    }
    if (aligned) {
#define BRR_SRC_CASE(KK) \
    case KK: launch_fixed_sweep<KK, false, SRC>(ctx, b, t_full, t_last, n_rolls, seed, out, stream); return;
        switch (k) {
            BRR_SRC_CASE(1) BRR_SRC_CASE(2) BRR_SRC_CASE(3) BRR_SRC_CASE(4)
            BRR_SRC_CASE(5) BRR_SRC_CASE(6) BRR_SRC_CASE(7) BRR_SRC_CASE(8)
            default: break;
        }
#undef BRR_SRC_CASE
    }
    launch_fixed_direct<SRC, false>(ctx, b, k, t_full, t_last, n_rolls, seed, out, stream);
}

brr_status launch_dice_fixed_src(brr_ctx *ctx, uint32_t source, uint32_t bm1, uint32_t k, uint64_t t_full,
                                 uint64_t t_last, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                                 cudaStream_t stream) {
    if (source == BRR_WORDS_SPLITMIX64)
        return launch_dice_fixed(ctx, bm1, k, t_full, t_last, n_rolls, seed, out, stream);
    if (n_rolls == 0) return BRR_OK;
    const bool full = bm1 == 0xFFFFFFFFu;
    const uint32_t b = bm1 + 1;  // unused (wraps to 0) when full
    const bool aligned = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    if (source == BRR_WORDS_CHACHA20)
        dispatch_fixed_src<BRR_WORDS_CHACHA20>(ctx, b, k, full, aligned, t_full, t_last, n_rolls, seed, out, stream);
    else
        dispatch_fixed_src<BRR_WORDS_SPLITMIX32>(ctx, b, k, full, aligned, t_full, t_last, n_rolls, seed, out,
                                                 stream);
    return cuda_status(cudaGetLastError());
}

}  // namespace brr
