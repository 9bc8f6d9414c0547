// words.cuh -- counter-based word sources other than the SplitMix64 stream,
// the Theorem 1 chain at L = 32, and the batch roll of a shuffle plan on any
// source (used by the swap-index and chain-resolution kernels).
//
// Section 7 runs the batched shuffle with generators of very different cost
// (Lehmer, PCG64, ChaCha) and finds that batching saves more the costlier a
// word is.  Those generators carry sequential state; here every source is a
// pure function of (seed, g, a) with the counter c = (g << 16) | a, so that
// batches and their retries stay independent:
//   BRR_WORDS_SPLITMIX64  word(seed, g, a) of brr_common.cuh, L = 64;
//   BRR_WORDS_CHACHA20    the first 64 bits of one 20-round ChaCha block
//                         (Bernstein 2008; input layout of RFC 8439): key =
//                         the seed's 8 bytes then 24 zero bytes, block
//                         counter = low 32 bits of c, nonce = (high 32 bits of
//                         c, 0, 0); the word is out[0] + 2^32 out[1], L = 64;
//   BRR_WORDS_SPLITMIX32  the high 32 bits of word(seed, g, a), L = 32 (the
//                         word size of Table 2's second column): every chain
//                         product is 32 x 32 bits and every batch product is
//                         at most 2^32.
#pragma once

#include "brr_common.cuh"

namespace brr {

__device__ __forceinline__ uint32_t rotl32(uint32_t x, uint32_t s) { return __funnelshift_l(x, x, s); }

// ChaCha quarter round on four state words.
__device__ __forceinline__ void chacha_qr(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t &d) {
    a += b; d = rotl32(d ^ a, 16);
    c += d; b = rotl32(b ^ c, 12);
    a += b; d = rotl32(d ^ a, 8);
    c += d; b = rotl32(b ^ c, 7);
}

// Word a of batch g from the ChaCha20 source: ten double rounds (a column
// round then a diagonal round) on the 4x4 state, then the input added back to
// the two output words that form the word.  The state lives in registers.
__device__ __forceinline__ uint64_t chacha20_word(uint64_t seed, uint64_t g, uint32_t a) {
    constexpr uint32_t s0 = 0x61707865u, s1 = 0x3320646eu, s2 = 0x79622d32u, s3 = 0x6b206574u;
    const uint64_t c = (g << 16) | a;
    uint32_t x0 = s0, x1 = s1, x2 = s2, x3 = s3;
    uint32_t x4 = (uint32_t)seed, x5 = (uint32_t)(seed >> 32), x6 = 0, x7 = 0;
    uint32_t x8 = 0, x9 = 0, x10 = 0, x11 = 0;
    uint32_t x12 = (uint32_t)c, x13 = (uint32_t)(c >> 32), x14 = 0, x15 = 0;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        chacha_qr(x0, x4, x8, x12);
        chacha_qr(x1, x5, x9, x13);
        chacha_qr(x2, x6, x10, x14);
        chacha_qr(x3, x7, x11, x15);
        chacha_qr(x0, x5, x10, x15);
        chacha_qr(x1, x6, x11, x12);
        chacha_qr(x2, x7, x8, x13);
        chacha_qr(x3, x4, x9, x14);
    }
    return (uint64_t)(x0 + s0) | ((uint64_t)(x1 + s1) << 32);
}

// Word a of batch g from the 32-bit source.
__device__ __forceinline__ uint32_t splitmix32_word(uint64_t seed, uint64_t g, uint32_t a) {
    return (uint32_t)(word(seed, g, a) >> 32);
}

// (die, r) <- b (*) r at L = 32: one 32x32->64 product; the die is its high
// word and the new leftover its low word.
__device__ __forceinline__ uint32_t chain_step32(uint32_t &r, uint32_t b) {
    const uint64_t p = (uint64_t)r * b;
    r = (uint32_t)p;
    return (uint32_t)(p >> 32);
}

// Lemire's threshold at L = 32: 2^32 mod B for 1 <= B <= 2^32 (0 for 2^32).
__device__ __forceinline__ uint32_t threshold32(uint64_t B) {
    if (B >= (1ull << 32)) return 0;
    const uint32_t b = (uint32_t)B;
    return (0u - b) % b;
}

// Batch g of a plan (Algorithm 4) with the words of source SRC: the chain
// at the source's word size, the fast test against the segment's bound u,
// the exact threshold 2^L mod B below it; map(i-1-m, a_m) for the k dice
// as roll_plan_batch does.  The SplitMix64 source is roll_plan_batch itself;
// the others are written as one loop so that the costly word function is
// inlined once.  Returns false if the attempt budget ran out.
template <uint32_t SRC, typename Map>
__device__ __forceinline__ bool roll_plan_batch_src(const Seg *segs, int nseg, uint64_t g, uint64_t seed,
                                                    Map map) {
    if constexpr (SRC == BRR_WORDS_SPLITMIX64) {
        return roll_plan_batch(segs, nseg, g, seed, map);
    } else {
        int s = 0;
        while (s + 1 < nseg && segs[s + 1].g0 <= g) s++;
        const Seg sg = segs[s];
        const uint32_t k = sg.k;
        const uint32_t i = sg.i0 - (uint32_t)(g - sg.g0) * k;
        uint32_t a[BRR_SCHED_KMAX];
        bool ok = true, have_t = false;
        uint64_t t = 0;
        for (uint32_t att = 0;;) {
            uint64_t left;
            if constexpr (SRC == BRR_WORDS_SPLITMIX32) {
                uint32_t r = splitmix32_word(seed, g, att);
#pragma unroll
                for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
                    if (m < k) a[m] = chain_step32(r, i - m);
                left = r;
            } else {
                uint64_t r = chacha20_word(seed, g, att);
#pragma unroll
                for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
                    if (m < k) a[m] = chain_step(r, i - m);
                left = r;
            }
            if (left >= sg.u) break;
            if (!have_t) {
                const uint64_t B = (uint64_t)falling(i, k);
                t = SRC == BRR_WORDS_SPLITMIX32 ? (uint64_t)threshold32(B) : (0 - B) % B;
                have_t = true;
            }
            if (left >= t) break;
            if (++att >= kMaxAttempts) { ok = false; break; }
        }
#pragma unroll
        for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
            if (m < k) map(i - 1 - m, a[m]);
        return ok;
    }
}

// Batches g_lo..g_hi-1 of a plan with the words of source SRC, one thread
// per batch, CTA-strided.
template <uint32_t SRC, typename Map>
__device__ void roll_plan_range_src(const Seg *segs, int nseg, uint64_t g_lo, uint64_t g_hi, uint64_t seed,
                                    int &err, Map map) {
    for (uint64_t g = g_lo + threadIdx.x; g < g_hi; g += blockDim.x)
        if (!roll_plan_batch_src<SRC>(segs, nseg, g, seed, map)) err = BRR_ERETRY;
}

}  // namespace brr
