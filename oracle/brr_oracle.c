/*
 * brr_oracle.c -- plain, sequential CPU oracle for batched ranged random
 * integer generation (Brackett-Rozinsky & Lemire, "Batched Ranged Random
 * Integer Generation", arXiv 2408.06213).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library calls, links or
 * includes this file; the two implementations share no code.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may use it.
 *
 * Everything here is written for obviousness, not speed: one thread, no
 * blocking, 128-bit products through unsigned __int128, and every function
 * follows the paper's algorithm step by step in the paper's order.
 *
 * Word source (not in the paper, which uses sequential-state generators): the
 * L=64 random words are drawn from a counter-based stream
 *     word(seed, g, a) = mix64(seed + GOLDEN * ((g << 16) | a))   (mod 2^64)
 * where g counts batches of one stream from 0 and a counts the attempts of
 * batch g from 0 (a < 2^16).  mix64 is the SplitMix64 output finalizer
 * (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014).  A batch that is rejected 2^16 times in a row returns
 * ORC_ERETRY (probability below 2^-65536 for any valid batch).
 *
 * Status codes: 0 ok, 1 invalid argument, 4 retry budget exhausted.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ERETRY 4

#define ORC_MAX_ATTEMPTS 65536u
#define ORC_KMAX_SCHED 8u

static const uint64_t ORC_GOLDEN = 0x9E3779B97F4A7C15ull;

int orc_dice_range(const uint32_t *bm1, const uint32_t *off, uint64_t g_lo, uint64_t g_hi,
                   uint64_t seed, uint32_t *out);
int orc_dice_fixed_range(uint64_t b, unsigned k, uint64_t n_rolls, uint64_t g_lo, uint64_t g_hi,
                         uint64_t seed, uint32_t *out);

/* ---------------------------------------------------------------- words -- */

/* SplitMix64 finalizer: xor-shift 30, multiply, xor-shift 27, multiply,
 * xor-shift 31 (constants from the published SplitMix64 definition). */
uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The counter-based word source described in the header comment. */
uint64_t orc_word(uint64_t seed, uint64_t g, uint64_t a)
{
    uint64_t c = (g << 16) | (a & 0xFFFFu);
    return orc_mix64(seed + ORC_GOLDEN * c);
}

/* ------------------------------------------------ full-width arithmetic -- */

/* x (*) y at word size L (Section 1.1 notation): 2^L * hi + lo = x * y,
 * 0 <= lo < 2^L.  Valid for x, y < 2^64 and 1 <= L <= 64. */
static void fullmul(unsigned L, uint64_t x, uint64_t y, uint64_t *hi, uint64_t *lo)
{
    u128 p = (u128)x * (u128)y;
    if (L == 64) {
        *hi = (uint64_t)(p >> 64);
        *lo = (uint64_t)p;
    } else {
        *hi = (uint64_t)(p >> L);
        *lo = (uint64_t)(p & (((u128)1 << L) - 1));
    }
}

/* Theorem 1 (Section 4): starting from r0, for i = 1..k perform
 * (a_i, r_i) <- b_i (*) r_{i-1}.  Writes a_1..a_k and returns r_k.
 * Requires r0 < 2^L and every b_i <= 2^L (b_i < 2^64 as a uint64). */
uint64_t orc_chain(unsigned L, const uint64_t *b, unsigned k, uint64_t r0, uint64_t *a)
{
    uint64_t r = r0;
    for (unsigned i = 0; i < k; i++) {
        uint64_t hi, lo;
        fullmul(L, b[i], r, &hi, &lo);
        a[i] = hi;
        r = lo;
    }
    return r;
}

/* The batch product prod(b_i) as a 128-bit integer; returns ORC_EINVAL if it
 * exceeds 2^L (Theorem 1 requires prod(b) <= 2^L) or a bound is 0. */
static int batch_product(unsigned L, const uint64_t *b, unsigned k, u128 *B)
{
    u128 W = (u128)1 << L;
    u128 p = 1;
    for (unsigned i = 0; i < k; i++) {
        if (b[i] == 0) return ORC_EINVAL;
        p *= (u128)b[i];            /* p <= 2^64 and b < 2^64: no overflow */
        if (p > W) return ORC_EINVAL;
    }
    *B = p;
    return ORC_OK;
}

/* Lemire's criterion threshold t = 2^L mod prod(b) (Section 2, Theorem 1). */
int orc_threshold(unsigned L, const uint64_t *b, unsigned k, uint64_t *t)
{
    u128 B;
    int st = batch_product(L, b, k, &B);
    if (st) return st;
    *t = (uint64_t)((((u128)1) << L) % B);
    return ORC_OK;
}

/* ------------------------------------------------- single rolls (Sec 2) -- */

/* Lemire's nearly-divisionless method (Lemma 1, Section 2) at L = 64 for one
 * bound 1 <= b <= 2^32, drawing the words of batch g in attempt order:
 * (x, y) <- b (*) r; if y < b, compute t = 2^64 mod b and redraw while y < t. */
int orc_lemire(uint64_t b, uint64_t seed, uint64_t g, uint64_t *out)
{
    if (b == 0 || b > (1ull << 32)) return ORC_EINVAL;
    uint64_t a = 0, x, y;
    fullmul(64, b, orc_word(seed, g, a), &x, &y);
    if (y < b) {
        uint64_t t = (0 - b) % b;          /* 2^64 mod b, as "-b % b" */
        while (y < t) {
            a++;
            if (a >= ORC_MAX_ATTEMPTS) return ORC_ERETRY;
            fullmul(64, b, orc_word(seed, g, a), &x, &y);
        }
    }
    *out = x;
    return ORC_OK;
}

/* ------------------------------------------------ batched rolls (Sec 5) -- */

/* Algorithm 3 (batched dice rolls, unknown threshold) at L = 64 with the
 * words of batch g: run the Theorem 1 chain; b <- prod(b_i); if r < b then
 * t <- 2^64 mod b and, while r < t, draw the next word and rerun the chain.
 * *attempts receives the number of words used (>= 1). */
int orc_roll_batch(const uint64_t *b, unsigned k, uint64_t seed, uint64_t g,
                   uint64_t *a, uint32_t *attempts)
{
    u128 B;
    int st = batch_product(64, b, k, &B);
    if (st) return st;
    uint32_t att = 0;
    uint64_t r = orc_chain(64, b, k, orc_word(seed, g, att), a);
    if ((u128)r < B) {
        uint64_t t = (uint64_t)((((u128)1) << 64) % B);
        while (r < t) {
            att++;
            if (att >= ORC_MAX_ATTEMPTS) return ORC_ERETRY;
            r = orc_chain(64, b, k, orc_word(seed, g, att), a);
        }
    }
    if (attempts) *attempts = att + 1;
    return ORC_OK;
}

/* Algorithm 2 (batched dice rolls, known threshold t): repeat { draw a word,
 * run the chain } until r >= t. */
static int roll_batch_known(const uint64_t *b, unsigned k, uint64_t t,
                            uint64_t seed, uint64_t g, uint64_t *a)
{
    for (uint32_t att = 0; att < ORC_MAX_ATTEMPTS; att++) {
        uint64_t r = orc_chain(64, b, k, orc_word(seed, g, att), a);
        if (r >= t) return ORC_OK;
    }
    return ORC_ERETRY;
}

/* Bulk dice with per-roll bounds b = bm1 + 1 (so 1 <= b <= 2^32), grouped
 * into batches in CSR form: batch g holds the rolls off[g] .. off[g+1]-1 and
 * uses the word stream of batch index g.  With off == NULL every roll is its
 * own batch (the unbatched, one-word-per-roll form, which Algorithm 3 with
 * k = 1 reduces to Lemire's method).  out[x] is the roll at position x. */
int orc_dice(const uint32_t *bm1, const uint32_t *off, uint64_t n_batches,
             uint64_t n_rolls, uint64_t seed, uint32_t *out)
{
    if (off) {
        if (off[0] != 0 || off[n_batches] != n_rolls) return ORC_EINVAL;
        for (uint64_t g = 0; g < n_batches; g++)
            if (off[g + 1] < off[g]) return ORC_EINVAL;
    } else if (n_batches != n_rolls) {
        return ORC_EINVAL;
    }
    return orc_dice_range(bm1, off, 0, n_batches, seed, out);
}

/* The batches g_lo .. g_hi-1 of orc_dice (same layout and word streams; the
 * CSR offsets are taken as valid).  Every batch depends only on its own index,
 * so disjoint ranges may be rolled by separate threads. */
int orc_dice_range(const uint32_t *bm1, const uint32_t *off, uint64_t g_lo, uint64_t g_hi,
                   uint64_t seed, uint32_t *out)
{
    uint64_t *b = NULL, *a = NULL;
    uint64_t cap = 0;
    int st = ORC_OK;
    for (uint64_t g = g_lo; g < g_hi && st == ORC_OK; g++) {
        uint64_t s = off ? off[g] : g;
        uint64_t e = off ? off[g + 1] : g + 1;
        uint64_t k = e - s;
        if (k > cap) {
            cap = k;
            free(b); free(a);
            b = malloc(cap * sizeof *b);
            a = malloc(cap * sizeof *a);
            if (!b || !a) { st = ORC_EINVAL; break; }
        }
        for (uint64_t i = 0; i < k; i++) b[i] = (uint64_t)bm1[s + i] + 1;
        st = orc_roll_batch(b, (unsigned)k, seed, g, a, NULL);
        if (st == ORC_OK)
            for (uint64_t i = 0; i < k; i++) out[s + i] = (uint32_t)a[i];
    }
    free(b); free(a);
    return st;
}

/* Bulk dice with one fixed bound 1 <= b <= 2^32 in batches of k (b^k <= 2^64):
 * batch g covers rolls g*k .. g*k+k-1; the last batch may hold fewer rolls.
 * The threshold of a full batch is known in advance (Algorithm 2). */
int orc_dice_fixed(uint64_t b, unsigned k, uint64_t n_rolls, uint64_t seed, uint32_t *out)
{
    if (k == 0) return ORC_EINVAL;
    return orc_dice_fixed_range(b, k, n_rolls, 0, (n_rolls + k - 1) / k, seed, out);
}

/* The batches g_lo .. g_hi-1 of orc_dice_fixed (out is the whole run's
 * output); disjoint ranges may be rolled by separate threads. */
int orc_dice_fixed_range(uint64_t b, unsigned k, uint64_t n_rolls, uint64_t g_lo, uint64_t g_hi,
                         uint64_t seed, uint32_t *out)
{
    if (b == 0 || b > (1ull << 32) || k == 0 || k > 64) return ORC_EINVAL;
    uint64_t bv[64], a[64];
    for (unsigned i = 0; i < k; i++) bv[i] = b;
    uint64_t t_full;
    int st = orc_threshold(64, bv, k, &t_full);
    if (st) return st;
    uint64_t n_batches = (n_rolls + k - 1) / k;
    if (g_hi > n_batches) g_hi = n_batches;
    for (uint64_t g = g_lo; g < g_hi; g++) {
        uint64_t s = g * k;
        unsigned kk = (unsigned)((n_rolls - s) < k ? (n_rolls - s) : k);
        uint64_t t = t_full;
        if (kk != k) {
            st = orc_threshold(64, bv, kk, &t);
            if (st) return st;
        }
        st = roll_batch_known(bv, kk, t, seed, g, a);
        if (st) return st;
        for (unsigned i = 0; i < kk; i++) out[s + i] = (uint32_t)a[i];
    }
    return ORC_OK;
}

/* ------------------------------------------------------ shuffle (Sec 6) -- */

/* Batch-size rule of the full shuffle (Section 6, Section 7): with n_k the
 * largest remaining count at which batches of k dice are used, the batch
 * size for a remaining count i is the largest k in 1..k_max with i <= n_k
 * (k = 1 is always allowed).  nk has ORC_KMAX_SCHED + 1 entries, index k. */
static unsigned k_rule(uint64_t i, const uint64_t *nk, unsigned k_max)
{
    unsigned k = 1;
    for (unsigned c = 2; c <= k_max; c++)
        if (i <= nk[c]) k = c;
    return k;
}

unsigned orc_k_rule(uint64_t i, const uint64_t *nk, unsigned k_max)
{
    return k_rule(i, nk, k_max);
}

/* A schedule is usable when 1 <= k_max <= 8 and every batch it can produce
 * has a falling-factorial product n_k (n_k - 1) ... (n_k - k + 1) <= 2^64. */
static int sched_valid(const uint64_t *nk, unsigned k_max)
{
    if (k_max < 1 || k_max > ORC_KMAX_SCHED) return 0;
    for (unsigned c = 2; c <= k_max; c++) {
        u128 p = 1;
        for (unsigned m = 0; m < c && nk[c] > m; m++) {
            p *= (u128)(nk[c] - m);
            if (p > ((u128)1 << 64)) return 0;
        }
    }
    return 1;
}

static void swap_elems(void *data, uint32_t eb, uint64_t x, uint64_t y)
{
    if (eb == 4) {
        uint32_t *d = data, t = d[x]; d[x] = d[y]; d[y] = t;
    } else {
        uint64_t *d = data, t = d[x]; d[x] = d[y]; d[y] = t;
    }
}

/* One step of Algorithm 4 (batched partial shuffle) with i elements left to
 * shuffle and batch size k, using the words of batch g: roll the dice
 * i, i-1, ..., i-k+1 with the Theorem 1 chain, accept under Lemire's criterion
 * for the product i(i-1)...(i-k+1) (upper bound u <- exact product, so the
 * shortcut of Section 5 is not used), then exchange z[i-1-m] and z[a_{m+1}]
 * for m = 0..k-1 in that order.  j[i-1-m] receives a_{m+1} when j != NULL. */
static int partial_shuffle_step(void *z, uint32_t eb, uint64_t i, unsigned k,
                                uint64_t seed, uint64_t g, uint32_t *j)
{
    uint64_t b[ORC_KMAX_SCHED], a[ORC_KMAX_SCHED];
    for (unsigned m = 0; m < k; m++) b[m] = i - m;
    int st = orc_roll_batch(b, k, seed, g, a, NULL);
    if (st) return st;
    for (unsigned m = 0; m < k; m++) {
        if (j) j[i - 1 - m] = (uint32_t)a[m];
        if (z) swap_elems(z, eb, i - 1 - m, a[m]);
    }
    return ORC_OK;
}

/* Full Fisher-Yates shuffle (Algorithm 1) driven by Algorithm 4 batches:
 * i <- n; while i > 1: k <- min(k_rule(i), i - 1); one Algorithm 4 step with
 * batch index g; g <- g + 1; i <- i - k.  The last batch therefore covers all
 * remaining dice, as in Section 6.  j (optional, n entries) receives the swap
 * index of every position p (j[p] in [0, p], j[0] = 0).  With k_max = 1 this
 * is the unbatched shuffle (one word per die, Lemire's method). */
int orc_shuffle(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                const uint64_t *nk, unsigned k_max, uint32_t *j)
{
    if ((elem_bytes != 4 && elem_bytes != 8) || n > 0xFFFFFFFFull) return ORC_EINVAL;
    if (!sched_valid(nk, k_max)) return ORC_EINVAL;
    if (j && n) j[0] = 0;
    uint64_t i = n, g = 0;
    while (i > 1) {
        unsigned k = k_rule(i, nk, k_max);
        if (k > i - 1) k = (unsigned)(i - 1);
        int st = partial_shuffle_step(data, elem_bytes, i, k, seed, g, j);
        if (st) return st;
        g++;
        i -= k;
    }
    return ORC_OK;
}


/* ---------------------------------------------- naive batched shuffle --
 * The paper's comparison method (Section 3, "Batched dice rolls", and its
 * appendix listing of the naive batched shuffle): a batch of k dice of sizes
 * i, i-1, ..., i-k+1 is one roll of a die with B = i (i-1) ... (i-k+1)
 * sides by Lemire's method, whose value v is then split into the dice by
 * remainders of successive quotients, least significant first: die i - m
 * gets v mod (i - m), then v <- v div (i - m) (mixed-radix digits, Lemma 2).
 * The batches follow the same plan as orc_shuffle (the schedule's k per
 * remaining count); the paper's naive_shuffle_2 is the schedule n_2 = 2^32,
 * k_max = 2.  Rolls use the attempt words of the batch, as everywhere here. */

/* Lemire's method (Lemma 1) for a bound 1 <= B < 2^64: x = floor(B r / 2^64)
 * is accepted when the low half y = B r mod 2^64 is >= 2^64 mod B (computed
 * only when y < B). */
static int lemire64(uint64_t B, uint64_t seed, uint64_t g, uint64_t *out)
{
    if (B == 0) return ORC_EINVAL;
    uint64_t a = 0, x, y;
    fullmul(64, B, orc_word(seed, g, a), &x, &y);
    if (y < B) {
        uint64_t t = (0 - B) % B;
        while (y < t) {
            a++;
            if (a >= ORC_MAX_ATTEMPTS) return ORC_ERETRY;
            fullmul(64, B, orc_word(seed, g, a), &x, &y);
        }
    }
    *out = x;
    return ORC_OK;
}

/* Dice of sizes i, i-1, ..., i-k+1 from v in [0, i (i-1) ... (i-k+1)),
 * least significant first: d[m] in [0, i - m). */
void orc_naive_digits(uint64_t v, uint64_t i, unsigned k, uint64_t *d)
{
    for (unsigned m = 0; m < k; m++) {
        d[m] = v % (i - m);
        v /= (i - m);
    }
}

int orc_naive_shuffle(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                      const uint64_t *nk, unsigned k_max, uint32_t *j)
{
    if ((elem_bytes != 4 && elem_bytes != 8) || n > 0xFFFFFFFFull) return ORC_EINVAL;
    if (!sched_valid(nk, k_max)) return ORC_EINVAL;
    if (j && n) j[0] = 0;
    uint64_t i = n, g = 0;
    while (i > 1) {
        unsigned k = k_rule(i, nk, k_max);
        if (k > i - 1) k = (unsigned)(i - 1);
        u128 B = 1;
        for (unsigned m = 0; m < k; m++) B *= (u128)(i - m);
        if (B >> 64) return ORC_EINVAL;  /* the product must fit the word */
        uint64_t v, d[ORC_KMAX_SCHED];
        int st = lemire64((uint64_t)B, seed, g, &v);
        if (st) return st;
        orc_naive_digits(v, i, k, d);
        for (unsigned m = 0; m < k; m++) {
            if (j) j[i - 1 - m] = (uint32_t)d[m];
            if (data) swap_elems(data, elem_bytes, i - 1 - m, d[m]);
        }
        g++;
        i -= k;
    }
    return ORC_OK;
}

/* Sequential application of a swap sequence (the exchange of Algorithm 1):
 * for p = n-1 down to 1, exchange A[p] and A[j[p]].  Requires j[p] <= p. */
int orc_apply_swaps(void *data, uint64_t n, uint32_t elem_bytes, const uint32_t *j)
{
    if (elem_bytes != 4 && elem_bytes != 8) return ORC_EINVAL;
    for (uint64_t p = n; p-- > 1;) {
        if (j[p] > p) return ORC_EINVAL;
        swap_elems(data, elem_bytes, p, j[p]);
    }
    return ORC_OK;
}

/* Many independent shuffles: array s occupies elements offsets[s] ..
 * offsets[s+1]-1 of data and is shuffled with its own seed seeds[s]. */
int orc_shuffle_batched(void *data, const uint64_t *offsets, uint64_t n_arrays,
                        uint32_t elem_bytes, const uint64_t *seeds,
                        const uint64_t *nk, unsigned k_max)
{
    for (uint64_t s = 0; s < n_arrays; s++) {
        if (offsets[s + 1] < offsets[s]) return ORC_EINVAL;
        char *base = (char *)data + offsets[s] * elem_bytes;
        int st = orc_shuffle(base, offsets[s + 1] - offsets[s], elem_bytes,
                             seeds[s], nk, k_max, NULL);
        if (st) return st;
    }
    return ORC_OK;
}

/* Partial Fisher-Yates sample: the first m steps of Algorithm 1 on the
 * identity array A[x] = x of length n, in Algorithm 4 batches that stop at
 * stop = max(n - m, 1): i <- n; while i > stop: k <- min(k_rule(i), i - stop).
 * out[q] = A[n-1-q] after the steps, q = 0..m-1 (selection order).  For m = n
 * the last value is what remains in A[0]. */
int orc_sample(uint64_t n, uint64_t m, uint64_t seed, const uint64_t *nk,
               unsigned k_max, uint32_t *out)
{
    if (n > 0xFFFFFFFFull || m > n) return ORC_EINVAL;
    if (!sched_valid(nk, k_max)) return ORC_EINVAL;
    if (m == 0) return ORC_OK;
    uint32_t *A = malloc(n * sizeof *A);
    if (!A) return ORC_EINVAL;
    for (uint64_t x = 0; x < n; x++) A[x] = (uint32_t)x;
    uint64_t stop = (n - m) > 1 ? (n - m) : 1;
    uint64_t i = n, g = 0;
    int st = ORC_OK;
    while (i > stop) {
        unsigned k = k_rule(i, nk, k_max);
        if (k > i - stop) k = (unsigned)(i - stop);
        st = partial_shuffle_step(A, 4, i, k, seed, g, NULL);
        if (st) break;
        g++;
        i -= k;
    }
    if (st == ORC_OK)
        for (uint64_t q = 0; q < m; q++) out[q] = A[n - 1 - q];
    free(A);
    return st;
}

/* ------------------------------------------------- other word sources --
 * Section 7 runs the shuffle with three generators of very different cost
 * (Lehmer, PCG64 and ChaCha) and finds the batched method gains most with the
 * costliest.  Sequential-state generators cannot be split across threads, so
 * the alternatives here are counter-based too, each a function of
 * (seed, g, a) with c = (g << 16) | a as in orc_word:
 *   source 0  SplitMix64 (orc_word), L = 64;
 *   source 1  ChaCha20 (Bernstein, "ChaCha, a variant of Salsa20", 2008), L =
 *             64: one 20-round block with the constants, key, block counter
 *             and nonce laid out as in RFC 8439: key = seed as 8 little-endian
 *             bytes then 24 zero bytes, counter word = low 32 bits of c,
 *             nonce = (high 32 bits of c, 0, 0); the word is the first 8
 *             keystream bytes read little-endian, out[0] + 2^32 out[1];
 *   source 2  the high 32 bits of orc_word, L = 32 (the word size of the
 *             L = 32 column of Table 2): chain products are 32 x 32 bits and
 *             every batch product is at most 2^32. */
#define ORC_SRC_SPLITMIX64 0u
#define ORC_SRC_CHACHA20 1u
#define ORC_SRC_SPLITMIX32 2u

static uint32_t rotl32(uint32_t x, unsigned s) { return (x << s) | (x >> (32u - s)); }

/* ChaCha quarter round on state words a, b, c, d. */
static void chacha_quarter(uint32_t *x, int a, int b, int c, int d)
{
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 16);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 12);
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 8);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 7);
}

/* The ChaCha block function: `rounds` rounds (an even number) alternating
 * column and diagonal rounds, then the input added word by word. */
void orc_chacha_block(const uint32_t in[16], unsigned rounds, uint32_t out[16])
{
    uint32_t x[16];
    memcpy(x, in, sizeof(x));
    for (unsigned r = 0; r < rounds; r += 2) {
        chacha_quarter(x, 0, 4, 8, 12);
        chacha_quarter(x, 1, 5, 9, 13);
        chacha_quarter(x, 2, 6, 10, 14);
        chacha_quarter(x, 3, 7, 11, 15);
        chacha_quarter(x, 0, 5, 10, 15);
        chacha_quarter(x, 1, 6, 11, 12);
        chacha_quarter(x, 2, 7, 8, 13);
        chacha_quarter(x, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + in[i];
}

/* The input block of source 1 for seed and counter c. */
void orc_chacha_input(uint64_t seed, uint64_t c, uint32_t in[16])
{
    static const uint32_t sigma[4] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u};
    memset(in, 0, 16 * sizeof(uint32_t));
    for (int i = 0; i < 4; i++) in[i] = sigma[i];
    in[4] = (uint32_t)seed;
    in[5] = (uint32_t)(seed >> 32);
    in[12] = (uint32_t)c;
    in[13] = (uint32_t)(c >> 32);
}

unsigned orc_src_bits(unsigned src) { return src == ORC_SRC_SPLITMIX32 ? 32u : 64u; }

/* Word a of batch g from source src (0 for an unknown source). */
uint64_t orc_word_src(unsigned src, uint64_t seed, uint64_t g, uint64_t a)
{
    if (src == ORC_SRC_SPLITMIX64) return orc_word(seed, g, a);
    if (src == ORC_SRC_SPLITMIX32) return orc_word(seed, g, a) >> 32;
    if (src == ORC_SRC_CHACHA20) {
        uint32_t in[16], out[16];
        orc_chacha_input(seed, (g << 16) | (a & 0xFFFFu), in);
        orc_chacha_block(in, 20, out);
        return (uint64_t)out[0] | ((uint64_t)out[1] << 32);
    }
    return 0;
}

/* Algorithm 3 at the source's word size L with the words of batch g: the
 * chain, then, while r < 2^L mod prod(b), the next word and the chain again.
 * (The exact threshold is formed for every attempt: the fast path of Section
 * 5 cannot change which words are accepted.) */
int orc_roll_batch_src(unsigned src, const uint64_t *b, unsigned k, uint64_t seed, uint64_t g,
                       uint64_t *a, uint32_t *attempts)
{
    if (src > ORC_SRC_SPLITMIX32) return ORC_EINVAL;
    const unsigned L = orc_src_bits(src);
    uint64_t t;
    int st = orc_threshold(L, b, k, &t);
    if (st) return st;
    for (uint32_t att = 0; att < ORC_MAX_ATTEMPTS; att++) {
        uint64_t r = orc_chain(L, b, k, orc_word_src(src, seed, g, att), a);
        if (r >= t) {
            if (attempts) *attempts = att + 1;
            return ORC_OK;
        }
    }
    return ORC_ERETRY;
}

/* A schedule is usable at word size L when 1 <= k_max <= 8 and every batch it
 * can produce has a falling-factorial product at most 2^L. */
static int sched_valid_L(const uint64_t *nk, unsigned k_max, unsigned L)
{
    if (k_max < 1 || k_max > ORC_KMAX_SCHED) return 0;
    for (unsigned c = 2; c <= k_max; c++) {
        u128 p = 1;
        for (unsigned m = 0; m < c && nk[c] > m; m++) {
            p *= (u128)(nk[c] - m);
            if (p > ((u128)1 << L)) return 0;
        }
    }
    return 1;
}

/* orc_shuffle with the words of source src: the same plan (k_rule clamped to
 * i - 1, batch index g counting from 0), the same exchanges, at the source's
 * word size.  n < 2^32 (the largest die, n, must fit the 32-bit word too). */
int orc_shuffle_src(unsigned src, void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                    const uint64_t *nk, unsigned k_max, uint32_t *j)
{
    if (src > ORC_SRC_SPLITMIX32) return ORC_EINVAL;
    if ((elem_bytes != 4 && elem_bytes != 8) || n > 0xFFFFFFFFull) return ORC_EINVAL;
    if (!sched_valid_L(nk, k_max, orc_src_bits(src))) return ORC_EINVAL;
    if (j && n) j[0] = 0;
    uint64_t i = n, g = 0;
    while (i > 1) {
        unsigned k = k_rule(i, nk, k_max);
        if (k > i - 1) k = (unsigned)(i - 1);
        uint64_t b[ORC_KMAX_SCHED], a[ORC_KMAX_SCHED];
        for (unsigned m = 0; m < k; m++) b[m] = i - m;
        int st = orc_roll_batch_src(src, b, k, seed, g, a, NULL);
        if (st) return st;
        for (unsigned m = 0; m < k; m++) {
            if (j) j[i - 1 - m] = (uint32_t)a[m];
            if (data) swap_elems(data, elem_bytes, i - 1 - m, a[m]);
        }
        g++;
        i -= k;
    }
    return ORC_OK;
}

/* Algorithm 2 (known threshold) with the words of source src: bulk dice of
 * one bound b in batches of k (the last batch may be shorter), batch g
 * drawing the attempt words of stream index g of that source until the
 * chain's leftover is at least 2^L mod b^k, L the source's word size.
 * Source 0 gives orc_dice_fixed. */
int orc_dice_fixed_src(unsigned src, uint64_t b, unsigned k, uint64_t n_rolls, uint64_t seed, uint32_t *out)
{
    if (src > ORC_SRC_SPLITMIX32) return ORC_EINVAL;
    if (b == 0 || b > (1ull << 32) || k == 0 || k > 64) return ORC_EINVAL;
    const unsigned L = orc_src_bits(src);
    uint64_t bv[64], a[64];
    for (unsigned i = 0; i < k; i++) bv[i] = b;
    uint64_t t_full;
    int st = orc_threshold(L, bv, k, &t_full);
    if (st) return st;
    uint64_t n_batches = (n_rolls + k - 1) / k;
    for (uint64_t g = 0; g < n_batches; g++) {
        uint64_t s0 = g * k;
        unsigned kk = (unsigned)((n_rolls - s0) < k ? (n_rolls - s0) : k);
        uint64_t t = t_full;
        if (kk != k) {
            st = orc_threshold(L, bv, kk, &t);
            if (st) return st;
        }
        uint32_t att = 0;
        for (;;) {
            if (att >= ORC_MAX_ATTEMPTS) return ORC_ERETRY;
            uint64_t r = orc_chain(L, bv, kk, orc_word_src(src, seed, g, att), a);
            if (r >= t) break;
            att++;
        }
        for (unsigned i = 0; i < kk; i++) out[s0 + i] = (uint32_t)a[i];
    }
    return ORC_OK;
}

/* Bulk dice with per-roll bounds (orc_dice) with the words of source src:
 * Algorithm 3 batch by batch (orc_roll_batch_src), batches in CSR form, or
 * one roll per batch with off == NULL.  Source 0 gives orc_dice. */
int orc_dice_src(unsigned src, const uint32_t *bm1, const uint32_t *off, uint64_t n_batches,
                 uint64_t n_rolls, uint64_t seed, uint32_t *out)
{
    if (src > ORC_SRC_SPLITMIX32) return ORC_EINVAL;
    if (off) {
        if (off[0] != 0 || off[n_batches] != n_rolls) return ORC_EINVAL;
        for (uint64_t g = 0; g < n_batches; g++)
            if (off[g + 1] < off[g]) return ORC_EINVAL;
    } else if (n_batches != n_rolls) {
        return ORC_EINVAL;
    }
    uint64_t *b = NULL, *a = NULL;
    uint64_t cap = 0;
    int st = ORC_OK;
    for (uint64_t g = 0; g < n_batches && st == ORC_OK; g++) {
        uint64_t s0 = off ? off[g] : g;
        uint64_t e = off ? off[g + 1] : g + 1;
        uint64_t k = e - s0;
        if (k > cap) {
            cap = k;
            free(b); free(a);
            b = malloc(cap * sizeof *b);
            a = malloc(cap * sizeof *a);
            if (!b || !a) { st = ORC_EINVAL; break; }
        }
        for (uint64_t i = 0; i < k; i++) b[i] = (uint64_t)bm1[s0 + i] + 1;
        st = orc_roll_batch_src(src, b, (unsigned)k, seed, g, a, NULL);
        if (st == ORC_OK)
            for (uint64_t i = 0; i < k; i++) out[s0 + i] = (uint32_t)a[i];
    }
    free(b); free(a);
    return st;
}

/* ------------------------------------------------ generic-L test hooks -- */

/* One Algorithm 4 step at word size L with an explicit word r0 and an
 * explicit fast-path bound u (any u >= the product; Section 6): rolls dice
 * i..i-k+1, and if r < u computes the exact product and its threshold.
 * Returns 1 and applies the k exchanges to z (uint64 elements) when the word
 * is accepted, 0 when it is rejected (z untouched), -1 on invalid input. */
int orc_partial_shuffle_word_L(unsigned L, uint64_t *z, uint64_t i, unsigned k,
                               uint64_t u, uint64_t r0, uint64_t *a)
{
    if (L < 1 || L > 64 || k < 1 || k > 64 || k > i) return -1;
    uint64_t b[64];
    for (unsigned m = 0; m < k; m++) b[m] = i - m;
    u128 B;
    if (batch_product(L, b, k, &B)) return -1;
    /* u must bound the product from above.  A product of exactly 2^64 has
     * threshold 0, so no uint64 u is needed for it: every word is accepted. */
    int full = B == ((u128)1 << 64);
    if (!full && (u128)u < B) return -1;
    uint64_t r = orc_chain(L, b, k, r0, a);
    int accept = 1;
    if (!full && r < u) {
        uint64_t t = (uint64_t)((((u128)1) << L) % B);
        accept = r >= t;
    }
    if (!accept) return 0;
    for (unsigned m = 0; m < k; m++) {
        uint64_t x = i - 1 - m, y = a[m], tmp = z[x];
        z[x] = z[y];
        z[y] = tmp;
    }
    return 1;
}

/* ------------------------------------------- batch-size cost model (6.1) -- */

/* Expected cost per die of batches of k dice at remaining count n
 * (Section 6.1): p1 = n^(k falling) / 2^L is the chance of computing the
 * product and threshold, p2 = (2^L mod b) / 2^L the chance of a reroll, and
 *   c_avg = ((c_rng + k) / (1 - p2) + (c_div + k - 1) p1) / k.
 * Returns HUGE_VAL when the product exceeds 2^L. */
double orc_cost_avg(unsigned k, uint64_t n, unsigned L, double c_rng, double c_div)
{
    if (k < 1 || n < k || L < 1 || L > 64) return HUGE_VAL;
    u128 W = (u128)1 << L, b = 1;
    for (unsigned m = 0; m < k; m++) {
        b *= (u128)(n - m);
        if (b > W) return HUGE_VAL;
    }
    double p1 = (double)b / (double)W;
    double p2 = (double)(W % b) / (double)W;
    return ((c_rng + k) / (1.0 - p2) + (c_div + k - 1) * p1) / k;
}

/* n_k (Section 6.1): the largest n such that batches of k are cheaper than
 * batches of k-1 for every array length from k up to n.  Scans upward and
 * gives up (returns 0) past n_limit. */
uint64_t orc_nk(unsigned k, unsigned L, double c_rng, double c_div, uint64_t n_limit)
{
    if (k < 2) return 0;
    for (uint64_t n = k; n <= n_limit; n++)
        if (!(orc_cost_avg(k, n, L, c_rng, c_div) < orc_cost_avg(k - 1, n, L, c_rng, c_div)))
            return n - 1;
    return 0;
}
