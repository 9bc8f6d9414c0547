// brr_common.cuh -- helpers shared by the brr CUDA kernels and their host
// launchers: the counter-based word source, the Theorem 1 chain step, the
// batch plan of a (partial) shuffle, device error recording and a bounded
// grid barrier for cooperative launches.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/brr.h"

namespace brr {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kMaxAttempts = 1u << 16;  // attempts per batch (counter field)
constexpr int kMaxSegs = 24;                 // segments of one shuffle plan

typedef unsigned __int128 u128;

// ------------------------------------------------------------ word source --
// SplitMix64 output finalizer (Steele, Lea & Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// word(seed, g, a): the a-th attempt word of batch g of one stream.
__host__ __device__ __forceinline__ uint64_t word(uint64_t seed, uint64_t g, uint32_t a) {
    return mix64(seed + kGolden * ((g << 16) | a));
}

// --------------------------------------------------- Theorem 1 chain steps --
// (a, r) <- b (*) r for a 32-bit bound b.  The 64x32 product is formed from
// 32-bit multiply-adds: the low half of r times b (low and high words), then
// the high half times b plus the first product's high word, with the carry
// of the low word taken into the high one (mad.lo.cc / madc.hi); the new r
// is (low word of the second, low word of the first) and the die is the
// second's high word.  (Measured a few percent faster than two 64-bit-wide
// multiply-adds, which need the carry-in widened into a register pair.)
__device__ __forceinline__ uint32_t chain_step(uint64_t &r, uint32_t b) {
    const uint32_t lo = (uint32_t)r, hi = (uint32_t)(r >> 32);
    const uint32_t p0lo = lo * b, p0hi = __umulhi(lo, b);
    uint32_t p1lo, p1hi;
    asm("mad.lo.cc.u32 %0, %2, %3, %4;\n\t"
        "madc.hi.u32 %1, %2, %3, 0;"
        : "=r"(p1lo), "=r"(p1hi)
        : "r"(hi), "r"(b), "r"(p0hi));
    r = ((uint64_t)p1lo << 32) | p0lo;
    return p1hi;
}

// The same step for a bound given as bm1 = b - 1, so that b = 2^32 is
// representable: b*r = bm1*r + r.  Both partial sums fit 64 bits:
// (2^32-1)^2 + 2(2^32-1) = 2^64 - 1.
__device__ __forceinline__ uint32_t chain_step_m1(uint64_t &r, uint32_t bm1) {
    const uint32_t lo = (uint32_t)r, hi = (uint32_t)(r >> 32);
    const uint64_t p0 = (uint64_t)lo * bm1 + lo;
    const uint64_t p1 = (uint64_t)hi * bm1 + ((uint64_t)hi + (p0 >> 32));
    r = (p1 << 32) | (uint32_t)p0;
    return (uint32_t)(p1 >> 32);
}

// ---------------------------------------- the same on 32-bit word halves --
// The per-roll-bound dice kernel keeps its words, counters and leftovers as
// two 32-bit registers (lo, hi): the 64-bit forms above make the compiler
// build register pairs and copy values into them, and those copies were a
// third of that kernel's instructions.

// z = mix64(x) for x = (xh:xl), result (zh:zl): each xor-shift is a funnel
// shift of the pair and a shift of the high word; each 64-bit multiply by a
// constant is the low-word product plus the two cross products' low words.
__device__ __forceinline__ void mix64_halves(uint32_t xl, uint32_t xh, uint32_t &zl, uint32_t &zh) {
    asm("{\n\t"
        ".reg .u32 t, u, l, h;\n\t"
        "shf.r.clamp.b32 t, %2, %3, 30;\n\t"
        "shr.u32 u, %3, 30;\n\t"
        "xor.b32 l, %2, t;\n\t"
        "xor.b32 h, %3, u;\n\t"
        "mul.hi.u32 t, l, 0x1CE4E5B9;\n\t"
        "mad.lo.u32 t, l, 0xBF58476D, t;\n\t"
        "mad.lo.u32 h, h, 0x1CE4E5B9, t;\n\t"
        "mul.lo.u32 l, l, 0x1CE4E5B9;\n\t"
        "shf.r.clamp.b32 t, l, h, 27;\n\t"
        "shr.u32 u, h, 27;\n\t"
        "xor.b32 l, l, t;\n\t"
        "xor.b32 h, h, u;\n\t"
        "mul.hi.u32 t, l, 0x133111EB;\n\t"
        "mad.lo.u32 t, l, 0x94D049BB, t;\n\t"
        "mad.lo.u32 h, h, 0x133111EB, t;\n\t"
        "mul.lo.u32 l, l, 0x133111EB;\n\t"
        "shf.r.clamp.b32 t, l, h, 31;\n\t"
        "shr.u32 u, h, 31;\n\t"
        "xor.b32 %0, l, t;\n\t"
        "xor.b32 %1, h, u;\n\t"
        "}"
        : "=r"(zl), "=r"(zh)
        : "r"(xl), "r"(xh));
}

// (xh:xl) += (ah:al) modulo 2^64.
__device__ __forceinline__ void add64_halves(uint32_t &xl, uint32_t &xh, uint32_t al, uint32_t ah) {
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+r"(xl), "+r"(xh) : "r"(al), "r"(ah));
}

// (a, r) <- (bm1 + 1) (*) r on halves, b = 2^32 included: b r = bm1 r + r,
// word by word -- word 0: lo(bm1 rl) + rl; word 1: hi(bm1 rl) + rh +
// lo(bm1 rh) + carry; word 2 (the die): hi(bm1 rh) + carries.  b r < 2^96,
// so the die fits 32 bits.
__device__ __forceinline__ uint32_t chain_step_m1_halves(uint32_t &rl, uint32_t &rh, uint32_t bm1) {
    uint32_t l0, t, d, l1;
    asm("mad.lo.cc.u32 %0, %4, %6, %4;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %5;\n\t"
        "madc.hi.u32 %2, %5, %6, 0;\n\t"
        "mad.lo.cc.u32 %3, %5, %6, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "=&r"(l0), "=&r"(t), "=&r"(d), "=&r"(l1)
        : "r"(rl), "r"(rh), "r"(bm1));
    rl = l0;
    rh = l1;
    return d;
}

// Running batch product kept as B - 1 so that B = 2^64 fits: multiplying by
// b = bm1 + 1 gives B' - 1 = (B-1)*bm1 + (B-1) + bm1.  Returns false when
// B' > 2^64 (the batch violates Theorem 1's condition).
__device__ __forceinline__ bool prod_m1_step(uint64_t &Bm1, uint32_t bm1) {
    const uint32_t lo = (uint32_t)Bm1, hi = (uint32_t)(Bm1 >> 32);
    const uint64_t q0 = (uint64_t)lo * bm1;
    const uint64_t q1 = (uint64_t)hi * bm1 + (q0 >> 32);
    if (q1 >> 32) return false;
    const uint64_t prod = (q1 << 32) | (uint32_t)q0;
    uint64_t s = prod + Bm1;
    bool ok = s >= prod;
    const uint64_t s2 = s + bm1;
    ok = ok && (s2 >= s);
    Bm1 = s2;
    return ok;
}

// Lemire's threshold t = 2^64 mod B (Section 2: accept a word iff its
// leftover is >= t) for 1 <= B < 2^64, exact.  Only reached on the rare path
// r < B, but for batch products close to 2^64 that path is common, so the
// software 64-bit remainder is avoided for B >= 2^43:
//  - B a power of two: t = 0;  B > 2^63: t = 2^64 - B (quotient 1);
//  - 2^62 < B < 2^63: the quotient is 3 if 3B < 2^64, else 2;
//  - 2^43 <= B < 2^62 (clz 2..20): the quotient Q = floor(2^64 / B) is below
//    2^22; q = trunc(2^64 / float(B)) has relative error below 5 * 2^-24
//    (rounding of B plus the <= 2 ulp of the fast division), so |q - Q| <= 1,
//    and c = 2^64 - q B (mod 2^64) lies in [0, B) for q = Q, in [B, 2B) for
//    q = Q - 1 and in [2^64 - B, 2^64) for q = Q + 1 -- ranges that do not
//    overlap when B < 2^62 -- which fixes t exactly;
//  - smaller B: the remainder "-B % B" (rare: r < B has probability B/2^64).
__device__ __forceinline__ uint64_t lemire_threshold(uint64_t B) {
    if ((B & (B - 1)) == 0) return 0;
    if (B > (1ull << 63)) return 0 - B;
    const int s = __clzll((long long)B);
    if (s == 1) return B <= 0x5555555555555555ull ? 0 - 3 * B : 0 - 2 * B;
    if (s > 20) return (0 - B) % B;
    const float qf = __fdividef(18446744073709551616.0f, __ull2float_rn(B));
    const uint64_t c = 0 - __float2ull_rz(qf) * B;
    if (c < B) return c;
    if (c < 2 * B) return c - B;
    return c + B;
}

// The same for a product held as B - 1 (so that B = 2^64 is representable;
// its threshold is 0).
__device__ __forceinline__ uint64_t threshold_from_m1(uint64_t Bm1) {
    if (Bm1 == ~0ull) return 0;
    return lemire_threshold(Bm1 + 1);
}

// ---------------------------------------------------------- shuffle plans --
// Batch-size rule (Section 6): the largest k in 1..k_max with i <= n_k[k].
__host__ __device__ __forceinline__ uint32_t k_rule(uint64_t i, const uint64_t *nk, uint32_t k_max) {
    uint32_t k = 1;
    for (uint32_t c = 2; c <= k_max; c++)
        if (i <= nk[c]) k = c;
    return k;
}

// i (i-1) ... (i-k+1) as a 128-bit value.
__host__ __device__ __forceinline__ u128 falling(uint64_t i, uint32_t k) {
    u128 p = 1;
    for (uint32_t m = 0; m < k && i > m; m++) p *= (u128)(i - m);
    return p;
}

// A schedule is usable at word size L (32 or 64) when 1 <= k_max <= 8 and
// every batch it can form has a product of at most 2^L (Theorem 1).
__host__ __device__ __forceinline__ bool sched_valid_bits(const uint64_t *nk, uint32_t k_max, uint32_t L) {
    if (k_max < 1 || k_max > BRR_SCHED_KMAX) return false;
    for (uint32_t c = 2; c <= k_max; c++) {
        u128 p = 1;
        for (uint32_t m = 0; m < c && nk[c] > m; m++) {
            p *= (u128)(nk[c] - m);
            if (p > ((u128)1 << L)) return false;
        }
    }
    return true;
}

__host__ __device__ __forceinline__ bool sched_valid(const uint64_t *nk, uint32_t k_max) {
    return sched_valid_bits(nk, k_max, 64);
}

struct Seg {
    uint64_t g0, count, u;
    uint32_t i0, k;
};

// Plan of a partial shuffle of n elements stopping at `stop` elements left:
// i <- n; while i > stop: k <- min(rule(i), i - stop); batch; i <- i - k.
// Runs of equal k are folded into segments: with K = rule(i) and no clamp,
// the rule stays K while i exceeds T = max{n_k[c] : K < c <= k_max}, so the
// batches i, i-k, i-2k, ... down to max(T+1, stop+k) form one segment.
// Returns the number of segments (or -1 if more than max_segs would be
// needed) and the number of batches in *n_batches.
__host__ __device__ inline int plan_segments(uint64_t n, uint64_t stop, const uint64_t *nk,
                                             uint32_t k_max, Seg *segs, int max_segs,
                                             uint64_t *n_batches) {
    uint64_t i = n, g = 0;
    int ns = 0;
    while (i > stop) {
        const uint32_t K = k_rule(i, nk, k_max);
        uint32_t k = K;
        if ((uint64_t)k > i - stop) k = (uint32_t)(i - stop);
        uint64_t count = 1;
        if (k == K) {
            uint64_t T = 0;
            for (uint32_t c = K + 1; c <= k_max; c++)
                if (nk[c] < i && nk[c] > T) T = nk[c];
            uint64_t min_i = T + 1;
            if (stop + k > min_i) min_i = stop + k;
            count = (i - min_i) / k + 1;
        }
        if (ns < max_segs) {
            segs[ns].g0 = g;
            segs[ns].count = count;
            segs[ns].u = (uint64_t)falling(i, k);  // < 2^64 for i < 2^32
            segs[ns].i0 = (uint32_t)i;
            segs[ns].k = k;
        }
        ns++;
        g += count;
        i -= count * k;
    }
    *n_batches = g;
    return ns <= max_segs ? ns : -1;
}

// Rolls batch g of a plan (Algorithm 4 with the Theorem 1 chain) and calls
// map(i-1-m, a_m) for its k dice i, i-1, ..., i-k+1: the swap target of
// position i-1-m.  The fast accept test compares the leftover word with the
// segment's bound u >= the product; only below it is the exact Lemire
// threshold formed.  Returns false if the attempt budget ran out (the
// targets of the last attempt are still passed to map).
template <typename Map>
__device__ __forceinline__ bool roll_plan_batch(const Seg *segs, int nseg, uint64_t g,
                                                uint64_t seed, Map map) {
    int s = 0;
    while (s + 1 < nseg && segs[s + 1].g0 <= g) s++;
    const Seg sg = segs[s];
    const uint32_t k = sg.k;
    const uint32_t i = sg.i0 - (uint32_t)(g - sg.g0) * k;
    uint32_t a[BRR_SCHED_KMAX];
    uint32_t att = 0;
    bool ok = true;
    uint64_t r = word(seed, g, 0);
#pragma unroll
    for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
        if (m < k) a[m] = chain_step(r, i - m);
    if (r < sg.u) {
        const uint64_t t = lemire_threshold((uint64_t)falling(i, k));
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
        if (m < k) map(i - 1 - m, a[m]);
    return ok;
}

// Rolls batches g_lo..g_hi-1 of a plan, one thread per batch, CTA-strided.
template <typename Map>
__device__ void roll_plan_range(const Seg *segs, int nseg, uint64_t g_lo, uint64_t g_hi,
                                uint64_t seed, int &err, Map map) {
    for (uint64_t g = g_lo + threadIdx.x; g < g_hi; g += blockDim.x)
        if (!roll_plan_batch(segs, nseg, g, seed, map)) err = BRR_ERETRY;
}

// ------------------------------------------------------ device error word --
__device__ __forceinline__ void record_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// bar[0] counts arrivals, bar[1] is the generation.  The wait is bounded:
// after `limit_ns` without the generation moving (or a spin count that the
// same time cannot take, should the timer stall), BRR_ETIMEOUT is recorded
// and false is returned.  Also returns false once any error is recorded, so
// that every block leaves its loop within one bounded wait.  `nblocks` is the
// number of arrivals that releases the barrier (the grid's block count).
constexpr uint64_t kBarrierLimitNs = 2000000000ull;  // 2 s

__device__ inline bool grid_barrier_bounded(uint32_t *bar, int *err, uint32_t nblocks, uint64_t limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t gen = ld_acquire_u32(&bar[1]);
        __threadfence();
        const uint32_t arrived = atomicAdd(&bar[0], 1u);
        int ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            // every spin includes a device-scope load and a sleep: far more
            // than 16 ns, so this count is only reached if the timer stalls
            const uint64_t max_spins = (limit_ns >> 4) + 65536;
            uint64_t spins = 0;
            while (ld_acquire_u32(&bar[1]) == gen) {
                if ((++spins & 63u) == 0) {
                    if (globaltimer_ns() - t0 > limit_ns || spins > max_spins) {
                        record_error(err, BRR_ETIMEOUT);
                        ok = 0;
                        break;
                    }
                    if (ld_relaxed_i32(err) != 0) {
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (ok && ld_relaxed_i32(err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ inline bool grid_barrier(uint32_t *bar, int *err) {
    return grid_barrier_bounded(bar, err, gridDim.x * gridDim.y * gridDim.z, kBarrierLimitNs);
}

}  // namespace brr
