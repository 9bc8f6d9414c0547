/*
 * brr.h -- batched ranged random integers on NVIDIA GB300 (sm_103a).
 *
 * A C ABI over hand-written CUDA kernels for the method of Brackett-Rozinsky
 * and Lemire, "Batched Ranged Random Integer Generation" (arXiv 2408.06213):
 * several unbiased dice rolls in [0, b_1) ... [0, b_k) are taken from one
 * 64-bit random word by a chain of full-width multiplications (Theorem 1,
 * Section 4), accepted under Lemire's criterion on the final leftover word
 * (Section 2, Algorithms 2 and 3), and used to drive the Fisher-Yates shuffle
 * (Algorithm 1) in batches (Algorithm 4, Section 6).
 *
 * Word source.  The paper draws words from sequential generators (Section 7);
 * here every word is a pure function of (seed, g, a):
 *     word(seed, g, a) = mix64(seed + 0x9E3779B97F4A7C15 * ((g << 16) | a))
 * (mod 2^64), mix64 being the SplitMix64 output finalizer, g the index of a
 * batch within one stream and a = 0, 1, ... its attempts.  Rejected batches
 * are therefore retried in any order without changing any result, and every
 * output is a deterministic function of the inputs: it is bit-identical to
 * the sequential algorithms of the paper run on this word stream.  A batch
 * rejected 2^16 times in a row (probability below 2^-65536) is an error.
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; they
 *    must stay valid until the work queued on `stream` completes.  Host
 *    pointers (schedules) are read before the call returns.
 *  - All work is queued asynchronously on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  The call returns once the work is queued.
 *  - Argument errors detectable on the host return BRR_EINVAL before anything
 *    is queued.  Errors found by a kernel (invalid device-resident input,
 *    retry budget exhausted, a bounded wait that ran out) are recorded in a
 *    sticky per-context word read by brr_last_device_error(); outputs of a
 *    call that recorded an error are unspecified, but no kernel reads or
 *    writes outside the buffers described here.
 *  - A context is bound to the device current at brr_create() and owns the
 *    scratch memory its calls need (grown on demand with cudaMalloc; see
 *    brr_reserve to size it ahead of stream capture).  One context must not
 *    be used from two host threads at once; calls on one context that use
 *    scratch are ordered by the caller's streams (use one context per
 *    concurrent stream).
 */
#ifndef BRR_H
#define BRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* Same type as cudaStream_t. */
typedef struct CUstream_st *brr_stream_t;

typedef enum brr_status {
    BRR_OK = 0,
    BRR_EINVAL = 1,   /* invalid argument or invalid device-resident input */
    BRR_ENOMEM = 2,   /* scratch allocation failed (no partial side effects) */
    BRR_ECUDA = 3,    /* a CUDA runtime call failed */
    BRR_ERETRY = 4,   /* a batch was rejected 2^16 times in a row */
    BRR_ETIMEOUT = 5, /* a bounded device-side wait ran out */
    BRR_ENODEV = 6    /* no usable CUDA device */
} brr_status;

typedef struct brr_ctx brr_ctx;

/* Largest batch size a shuffle schedule may use (Table 2 lists k <= 8). */
#define BRR_SCHED_KMAX 8

/*
 * Batch-size schedule of a shuffle (Section 6, "Batch sizes"; Table 2).
 * With i elements still to shuffle, a batch rolls k dice where k is the
 * largest value in 1..k_max with i <= n_k[k] (k = 1 always qualifies); the
 * last batch is cut to the dice that remain.  n_k[0] and n_k[1] are ignored.
 * Valid when 1 <= k_max <= BRR_SCHED_KMAX and n_k[k] (n_k[k]-1) ...
 * (n_k[k]-k+1) <= 2^64 for every k in 2..k_max (so every batch product fits
 * the 64-bit word, as Theorem 1 requires).  k_max = 1 is the unbatched form:
 * one word per die, which is Lemire's method (Section 2).
 */
typedef struct brr_schedule {
    uint64_t n_k[BRR_SCHED_KMAX + 1];
    uint32_t k_max;
} brr_schedule;

/* The schedule of the paper's experiments (Section 7): n_2..n_6 = 2^30,
 * 2^19, 2^14, 2^11, 2^9 -- Table 2's L = 64 estimates rounded down to powers
 * of two -- and k_max = 6.  Passing NULL wherever a schedule is taken means
 * this schedule. */
void brr_schedule_paper(brr_schedule *s);

/* One segment of a shuffle plan: batches g0 .. g0 + count - 1 each roll k
 * dice; batch g0 + c rolls the dice i0 - c*k, i0 - c*k - 1, ...,
 * i0 - c*k - k + 1.  u = i0 (i0-1) ... (i0-k+1) bounds every product of the
 * segment from above (the upper bound u of Algorithm 4, Section 6). */
typedef struct brr_segment {
    uint64_t g0;
    uint64_t count;
    uint64_t u;
    uint32_t i0;
    uint32_t k;
} brr_segment;

/*
 * Host-only planning (no device work, usable without a GPU).  Describes the
 * batches of a partial Fisher-Yates shuffle of n elements that stops when
 * `stop` elements remain (stop = 1 for a full shuffle, Algorithm 1; stop =
 * max(n - m, 1) for a sample of m): i <- n; while i > stop: k <- min(rule(i),
 * i - stop); batch; i <- i - k (Algorithm 4 repeated, Section 6).
 * Writes at most max_segs segments to segs (may be NULL when max_segs = 0),
 * the number needed to *n_segs and the number of batches to *n_batches.
 * Returns BRR_EINVAL for an invalid schedule, n >= 2^32 or stop > max(n, 1).
 */
brr_status brr_shuffle_plan(uint64_t n, uint64_t stop, const brr_schedule *sched,
                            brr_segment *segs, uint32_t max_segs,
                            uint32_t *n_segs, uint64_t *n_batches);

/* Human-readable name of a status code (static storage). */
const char *brr_status_str(brr_status s);

/* Version string of the library (static storage). */
const char *brr_version(void);

/* Create a context on the current CUDA device.  BRR_ENODEV without one. */
brr_status brr_create(brr_ctx **ctx);

/* Release a context and its scratch (synchronises the device first). */
brr_status brr_destroy(brr_ctx *ctx);

/*
 * Wait for the work queued on `stream`, then return and clear the first
 * error any kernel of this context recorded since the last call (BRR_OK if
 * none).  Errors recorded by work on other streams are visible once that
 * work has completed.
 */
brr_status brr_last_device_error(brr_ctx *ctx, brr_stream_t stream);

/*
 * Grow the context's scratch so that shuffles of up to max_shuffle_len
 * elements (one array, or batched arrays of at most that length, either
 * swap method) and samples of up to max_sample_m draws run without
 * allocating, and set up the shuffle kernels' launch attributes.
 * Synchronous.  Needed before capturing calls into a CUDA graph: a call
 * whose scratch would have to grow while its stream is being captured
 * returns BRR_EINVAL and queues nothing.  Two optional parts of a batched
 * call are not covered: its size-class lists (36 bytes per array) and, when
 * arrays exceed the limit of the windows that stage whole, one 128 KiB
 * target slot per SM.  Outside capture the call grows the scratch for them;
 * during capture it goes without them (same output, more time).
 */
brr_status brr_reserve(brr_ctx *ctx, uint64_t max_shuffle_len, uint64_t max_sample_m);

/*
 * Bulk dice with per-roll bounds (Algorithm 3, "unknown threshold").
 *  bm1_dev    [n_rolls] uint32: roll x has bound b = bm1_dev[x] + 1, so
 *             1 <= b <= 2^32.
 *  batch_off_dev [n_batches + 1] uint32, nondecreasing, first 0, last
 *             n_rolls: batch g holds rolls batch_off_dev[g] ..
 *             batch_off_dev[g+1] - 1 and draws the words of stream index g.
 *             The product of a batch's bounds must be <= 2^64 (Theorem 1).
 *             NULL means one roll per batch (n_batches must equal n_rolls):
 *             the unbatched form, where each roll is Lemire's method.
 *  out_dev    [n_rolls] uint32: out_dev[x] in [0, b) is the roll at x.
 * Requires n_rolls < 2^32 and n_batches <= 2^32 - 64.  A batch whose
 * product exceeds 2^64, or offsets
 * that are not as described, record BRR_EINVAL on the device.
 */
brr_status brr_dice(brr_ctx *ctx, const uint32_t *bm1_dev, const uint32_t *batch_off_dev,
                    uint64_t n_batches, uint64_t n_rolls, uint64_t seed,
                    uint32_t *out_dev, brr_stream_t stream);

/*
 * Bulk dice with one bound b (1 <= b <= 2^32) in batches of k (1 <= k <= 64,
 * b^k <= 2^64): batch g covers rolls g*k .. g*k + k - 1 (the last batch may
 * be shorter) with the threshold 2^64 mod b^k computed once on the host
 * (Algorithm 2, "known threshold").  out_dev [n_rolls] uint32.  k = 1 is the
 * unbatched form.  Requires n_rolls < 2^40.
 */
brr_status brr_dice_fixed(brr_ctx *ctx, uint64_t b, uint32_t k, uint64_t n_rolls,
                          uint64_t seed, uint32_t *out_dev, brr_stream_t stream);

/*
 * Fisher-Yates shuffle (Algorithm 1) of n elements of elem_bytes (4 or 8)
 * bytes in place, with dice rolled in batches by `sched` (Algorithm 4; NULL
 * = the paper's schedule).  Batch g of the plan (brr_shuffle_plan with stop
 * = 1) draws the words of stream index g; die i - m of a batch gives the
 * swap index j[i-1-m].  The result is the permutation the sequential
 * algorithm produces: for p = n-1 down to 1, exchange A[p] and A[j[p]].
 *  j_out_dev  optional [n] uint32 (may be NULL): receives j[p] in [0, p],
 *             j[0] = 0.
 *  data_dev   may be NULL when j_out_dev is not: then only the swap indices
 *             are generated (one thread per batch; for callers that apply
 *             them themselves, and to time the dice alone).
 * Requires n < 2^32.  Arrays above 65,536 elements use context scratch of
 * 8 + elem_bytes bytes per element (chain resolution; 24 with
 * BRR_SWAP_ROUNDS).
 */
brr_status brr_shuffle(brr_ctx *ctx, void *data_dev, uint64_t n, uint32_t elem_bytes,
                       uint64_t seed, const brr_schedule *sched, uint32_t *j_out_dev,
                       brr_stream_t stream);

/*
 * The naive batched shuffle, the paper's division-based comparison method
 * (Section 3, "Batched dice rolls", and the appendix's naive batched
 * shuffle): the k dice of a batch come from one Lemire roll v of their
 * product B = i (i-1) ... (i-k+1), split into dice by remainders of
 * successive quotients, least significant first (die i - m gets v mod
 * (i - m), then v <- v div (i - m)).  Batches follow the plan of `sched`
 * (NULL: brr_schedule_naive2, the paper's naive_shuffle_2) and use the words
 * of stream index g as brr_shuffle does; for the same batch the drawn value
 * v is the one brr_shuffle's chain draws, in the other digit order, so the
 * permutations differ.  Swap application as set by brr_set_swap_method.
 * data_dev = NULL with j_out_dev given: the swap indices only.
 * Scratch: as brr_shuffle on the grid path, plus 4 B per element when
 * j_out_dev is NULL.  Otherwise as brr_shuffle.
 */
brr_status brr_shuffle_naive(brr_ctx *ctx, void *data_dev, uint64_t n, uint32_t elem_bytes,
                             uint64_t seed, const brr_schedule *sched, uint32_t *j_out_dev,
                             brr_stream_t stream);

/* The schedule of the paper's naive_shuffle_2: single dice while more than
 * 2^32 elements remain, pairs below (n_2 = 2^32, k_max = 2). */
void brr_schedule_naive2(brr_schedule *s);

/*
 * Counter-based word sources of brr_shuffle_words.  Section 7 times the
 * batched shuffle with generators of different cost (Lehmer, PCG64, ChaCha)
 * and finds the gain from batching grows with the cost of a word.  Each
 * source here is a pure function of (seed, g, a), c = (g << 16) | a:
 *  BRR_WORDS_SPLITMIX64  word(seed, g, a) above; L = 64 (brr_shuffle's words)
 *  BRR_WORDS_CHACHA20    the first 8 bytes, little-endian, of one 20-round
 *                        ChaCha block (RFC 8439 layout): key = seed as 8
 *                        little-endian bytes then 24 zero bytes, block
 *                        counter = low 32 bits of c, nonce = high 32 bits of
 *                        c then 8 zero bytes; L = 64
 *  BRR_WORDS_SPLITMIX32  the high 32 bits of word(seed, g, a); L = 32: the
 *                        chain multiplies 32-bit words (Theorem 1 at L = 32)
 *                        and every batch product must be at most 2^32
 */
typedef enum {
    BRR_WORDS_SPLITMIX64 = 0,
    BRR_WORDS_CHACHA20 = 1,
    BRR_WORDS_SPLITMIX32 = 2
} brr_word_source;

/*
 * brr_dice with the words of `source` (brr_word_source): batch g draws the
 * words of stream index g of that source and is accepted under Algorithm 3
 * at the source's word size L.  Arguments, layout and errors as brr_dice,
 * except that at L = 32 (BRR_WORDS_SPLITMIX32) every batch product must be
 * at most 2^32 (a larger one records BRR_EINVAL on the device).
 * BRR_WORDS_SPLITMIX64 gives brr_dice's output.
 */
brr_status brr_dice_words(brr_ctx *ctx, uint32_t source, const uint32_t *bm1_dev, const uint32_t *batch_off_dev,
                          uint64_t n_batches, uint64_t n_rolls, uint64_t seed, uint32_t *out_dev,
                          brr_stream_t stream);

/*
 * brr_dice_fixed with the words of `source` (brr_word_source): batch g of k
 * dice draws the words of stream index g of that source, the Theorem 1 chain
 * runs at the source's word size L, and a batch is accepted when its
 * leftover is at least 2^L mod b^k (Algorithm 2).  For sources other than
 * SplitMix64: 1 <= k <= 8 and b^k <= 2^L (L = 32 for BRR_WORDS_SPLITMIX32),
 * else BRR_EINVAL; b = 2^32 is allowed where b^k fits.  out_dev [n_rolls]
 * uint32, n_rolls < 2^40.  BRR_WORDS_SPLITMIX64 is brr_dice_fixed itself.
 */
brr_status brr_dice_fixed_words(brr_ctx *ctx, uint32_t source, uint64_t b, uint32_t k, uint64_t n_rolls,
                                uint64_t seed, uint32_t *out_dev, brr_stream_t stream);

/*
 * brr_shuffle_batched with the words of `source` (brr_word_source): array s
 * is shuffled exactly as brr_shuffle_words would with seed seeds_dev[s].
 * sched NULL: the source's default schedule (as brr_shuffle_words).  The
 * swaps are applied by chain resolution whatever the context's swap method.
 * Arguments, layout and errors as brr_shuffle_batched.
 */
brr_status brr_shuffle_batched_words(brr_ctx *ctx, uint32_t source, void *data_dev, const uint64_t *offsets_dev,
                                     uint32_t n_arrays, uint32_t elem_bytes, const uint64_t *seeds_dev,
                                     uint64_t max_len, const brr_schedule *sched, brr_stream_t stream);

/* The L = 32 schedule: Table 2's L = 32 estimates (20,724, 581, 109) rounded
 * down to powers of two as Section 7 does for L = 64: n_2 = 2^14, n_3 = 2^9,
 * n_4 = 2^6, k_max = 4. */
void brr_schedule_l32(brr_schedule *s);

/*
 * brr_shuffle with the words of `source` (brr_word_source): the same plan,
 * batch g drawing the words of stream index g of that source, the same
 * Theorem 1 chain at the source's word size L with the acceptance test on
 * the leftover (2^L mod B, Section 2), and the same exchanges.  sched NULL:
 * the paper's schedule for L = 64 sources, brr_schedule_l32 for L = 32.  A
 * schedule whose batch products can exceed 2^L returns BRR_EINVAL.
 * BRR_WORDS_SPLITMIX64 is brr_shuffle itself.  For the other sources the swap
 * indices come from their own kernel and are applied by the context's swap
 * method (grid-wide chain resolution or rounds); scratch as brr_shuffle_naive.
 * data_dev = NULL with j_out_dev given: the swap indices only.
 */
brr_status brr_shuffle_words(brr_ctx *ctx, uint32_t source, void *data_dev, uint64_t n,
                             uint32_t elem_bytes, uint64_t seed, const brr_schedule *sched,
                             uint32_t *j_out_dev, brr_stream_t stream);

/*
 * How brr_shuffle and brr_shuffle_batched apply the swap sequence j[] to
 * the array.  Both give the sequential algorithm's permutation bit for bit;
 * they differ in speed only.
 *  BRR_SWAP_ROUNDS  deterministic-reservation rounds: every pending swap p
 *                   reserves slots p and j[p] by atomicMax on its priority
 *                   and commits when it holds both (about 3 log2 n rounds).
 *  BRR_SWAP_CHAINS  chain resolution: the steps are grouped by target in
 *                   sorted lists, and each final element is found by
 *                   following parent links (four parallel passes).
 *  BRR_SWAP_AUTO    the library's choice (currently chain resolution).
 */
typedef enum {
    BRR_SWAP_AUTO = 0,
    BRR_SWAP_ROUNDS = 1,
    BRR_SWAP_CHAINS = 2
} brr_swap_method;

/* Select the swap-application method of later shuffles on this context
 * (BRR_EINVAL for an unknown method).  Not thread-safe against shuffles
 * being queued on the same context. */
brr_status brr_set_swap_method(brr_ctx *ctx, uint32_t method);

/*
 * Kernel routing of chain-resolution shuffles and fixed-bound dice.  Every
 * setting gives the same result; they trade latency against throughput and
 * are what an autotuner (paper_2408_06213_gb300.tune) measures and sets.
 *  BRR_TUNE_SINGLE_CTA_MAX     brr_shuffle: arrays up to this length (at most
 *                              65,536) run in one CTA's shared memory
 *                              (default 4096); longer ones in four grid-wide
 *                              passes
 *  BRR_TUNE_SMALL_MAX          brr_shuffle_batched size classes: arrays up
 *  BRR_TUNE_MEDIUM_MAX         to SMALL_MAX elements run in 128-thread CTAs
 *                              (default 2048), up to MEDIUM_MAX in 256-thread
 *                              CTAs (default 8192), longer ones in 1024-thread
 *                              CTAs (up to 65,536 elements; beyond that one
 *                              CTA per array in global memory); at most 65,536
 *  BRR_TUNE_GRID_COOPERATIVE   brr_shuffle on the grid: 1 (default) = one
 *                              cooperative launch (lowest latency; it holds
 *                              the whole GPU while it runs); 0 = one launch
 *                              per pass, which can share the GPU with work on
 *                              other streams
 *  BRR_TUNE_FIXED_SWEEP        brr_dice_fixed: 1 (default) = a warp rolls
 *                              attempt 0 of every batch of its tile, then
 *                              sweeps the rejected ones from a compacted
 *                              queue; 0 = every lane owns fixed batches and
 *                              retries them in place
 *  BRR_TUNE_ORDERED_PUSH       chain-resolution shuffles in one CTA (batched
 *                              arrays up to 65,536 elements, and single
 *                              arrays up to SINGLE_CTA_MAX): 1 = the CTA
 *                              rolls its batches in rounds of one batch per
 *                              thread with a barrier between rounds, so that
 *                              pushes onto one target's list from different
 *                              rounds arrive in sequential order and fewer
 *                              lists need sorting; 0 (default; measured
 *                              faster on the 65,536-array layout) = no
 *                              barriers
 *  BRR_TUNE_WINDOW_ROUTE       brr_shuffle_batched with chain resolution:
 *                              1 (default) = the small class and the large
 *                              arrays that fit one CTA's shared memory whole
 *                              apply their swaps by deterministic
 *                              reservations over windows of consecutive
 *                              steps (one step per thread, a few rounds per
 *                              window), the rest by chain resolution; 0 =
 *                              chain resolution for every array
 */
typedef enum {
    BRR_TUNE_SINGLE_CTA_MAX = 1,
    BRR_TUNE_SMALL_MAX = 2,
    BRR_TUNE_MEDIUM_MAX = 3,
    BRR_TUNE_GRID_COOPERATIVE = 4,
    BRR_TUNE_FIXED_SWEEP = 5,
    BRR_TUNE_ORDERED_PUSH = 6,
    BRR_TUNE_WINDOW_ROUTE = 7
} brr_tune_param;

/* Set / read a routing parameter of this context (BRR_EINVAL for an unknown
 * parameter or value). */
brr_status brr_tune(brr_ctx *ctx, uint32_t param, uint64_t value);
brr_status brr_tune_get(brr_ctx *ctx, uint32_t param, uint64_t *value);

/*
 * Many independent shuffles in one launch sequence: array s holds elements
 * offsets_dev[s] .. offsets_dev[s+1] - 1 of data_dev (element offsets,
 * nondecreasing) and is shuffled exactly as brr_shuffle would with seed
 * seeds_dev[s].  max_len must bound every array's length (< 2^32); arrays
 * longer than max_len record BRR_EINVAL and are left untouched.
 */
brr_status brr_shuffle_batched(brr_ctx *ctx, void *data_dev, const uint64_t *offsets_dev,
                               uint32_t n_arrays, uint32_t elem_bytes,
                               const uint64_t *seeds_dev, uint64_t max_len,
                               const brr_schedule *sched, brr_stream_t stream);

/*
 * Partial Fisher-Yates sample (sampling is the application Section 8 names
 * as future work): the first m steps of Algorithm 1 on the identity array
 * A[x] = x of length n, in batches planned with stop = max(n - m, 1).
 * out_dev [m] uint32 receives A[n-1], A[n-2], ..., A[n-m] after those steps
 * (selection order), m distinct values in [0, n).  n is never materialised.
 * Requires m <= n < 2^32 and m <= 2^20.
 */
brr_status brr_sample(brr_ctx *ctx, uint64_t n, uint32_t m, uint64_t seed,
                      const brr_schedule *sched, uint32_t *out_dev, brr_stream_t stream);

/*
 * Many samples in one launch: request r draws m_dev[r] values from
 * [0, n_dev[r]) with seed seeds_dev[r] exactly as brr_sample would, into
 * out_dev[out_off_dev[r] ...].  max_m must bound every m_dev[r] (<= 2^20);
 * requests that violate it or m > n record BRR_EINVAL and are skipped.
 */
brr_status brr_sample_batched(brr_ctx *ctx, const uint64_t *n_dev, const uint32_t *m_dev,
                              const uint64_t *seeds_dev, const uint64_t *out_off_dev,
                              uint32_t n_req, uint32_t max_m, const brr_schedule *sched,
                              uint32_t *out_dev, brr_stream_t stream);

/*
 * Measured costs of the operations the batch-size cost model of Section 6.1
 * counts (that model picks the thresholds n_k of a schedule).  Writes four
 * figures to ns_per_op (host memory): nanoseconds of GPU time per operation
 * when every thread of a full grid runs it in registers, for
 *  [0] one random word (the SplitMix64 counter stream),
 *  [1] one Theorem 1 chain step (the model's multiplication, one die),
 *  [2] the exact threshold 2^64 mod B for B in [2^48, 2^64),
 *  [3] the same for B in [2^8, 2^40) (64-bit remainder).
 * The model's c_rng is [0]/[1] and c_div is [2]/[1] (or [3]/[1]).  Runs
 * and synchronises `stream`; about a millisecond of GPU time.
 */
brr_status brr_calibrate(brr_ctx *ctx, double *ns_per_op, brr_stream_t stream);

/* Largest shuffle brr_shuffle_noalloc accepts. */
#define BRR_NOALLOC_MAX_N (1u << 20)

/*
 * brr_shuffle without any device allocation (the paper has no counterpart:
 * this serves callers of the library, not the method).  Some callers cannot
 * allocate device memory on demand: code whose device memory is owned by
 * another allocator or capped by a fixed budget, and latency-critical loops
 * that cannot afford the device-wide synchronisation cudaMalloc / cudaFree
 * may imply.  This entry point takes no context and calls no cudaMalloc,
 * cudaFree or allocating library routine.  Its scratch (reservation words,
 * pending lists, swap indices; 24 bytes per position) is a fixed array of
 * about 24 MiB inside the library, which every GPU that loads the library
 * holds until the process exits.
 *  data_dev, n, elem_bytes, seed, sched, j_out_dev: as for brr_shuffle;
 *             the result is bit-identical to brr_shuffle's.
 *  status_dev optional device int (may be NULL): receives BRR_OK or the
 *             error a kernel recorded (BRR_ERETRY, BRR_ETIMEOUT) once the
 *             queued work has run.
 * Returns BRR_EINVAL for n > BRR_NOALLOC_MAX_N (use brr_shuffle for larger
 * arrays) and for the argument errors of brr_shuffle.  The first call on each
 * device looks up the device address of the fixed array (cudaGetSymbolAddress
 * with that device current); make that first call before any stream capture.
 * The address is kept for the life of the process: resetting a device
 * (cudaDeviceReset, or a reset of its primary context) after the first call
 * is not supported, since the array may then reload at another address.
 * Every call uses the same array, whatever its stream: calls whose work can
 * overlap on the GPU race with each other and must be ordered by the caller
 * (one stream, or events).  Each call clears the parts of the array that must
 * start at zero.
 */
brr_status brr_shuffle_noalloc(void *data_dev, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                               const brr_schedule *sched, uint32_t *j_out_dev, int *status_dev,
                               brr_stream_t stream);

/*
 * Self-test hook: t_dev[x] = 2^64 mod B_dev[x] (Lemire's threshold, Section
 * 2) as computed by the device routine every kernel uses on its rare path
 * (0 where B_dev[x] = 0).  Lets a test compare that routine with exact
 * arithmetic directly, since a wrong threshold changes only a tiny fraction
 * of outputs.  [n] uint64 device buffers owned by the caller.
 */
brr_status brr_selftest_threshold(const uint64_t *B_dev, uint64_t *t_dev, uint64_t n,
                                  brr_stream_t stream);

/*
 * Test hook for failure detection (the paper has no counterpart): the number
 * of attempts (words) a bulk-dice batch of this context may use before the
 * call records BRR_ERETRY, 1 .. 2^16 (the default, at which a valid batch
 * runs out with probability below 2^-65536).  Lowering it lets a test make
 * a high-rejection workload (one bound of 2^31 + 1 in pairs rejects a
 * quarter of its words) exhaust the budget on purpose; the rolls of such
 * batches are then not valid.  Applies to brr_dice, brr_dice_fixed and
 * their other-word-source forms.  BRR_EINVAL outside the range.
 */
brr_status brr_selftest_attempt_limit(brr_ctx *ctx, uint32_t limit);

/*
 * Self-test of failure detection (the paper has no counterpart): runs the
 * bounded grid-wide barrier that the cooperative shuffle kernels use, in one
 * block that waits for an arrival that never comes.  The wait gives up after
 * limit_ns (1 us .. 100 ms, else BRR_EINVAL) and records BRR_ETIMEOUT in the
 * context's device error word, which brr_last_device_error then returns; the
 * kernel ends and the context stays usable.  Uses 8 bytes of context scratch.
 */
brr_status brr_selftest_barrier_timeout(brr_ctx *ctx, uint64_t limit_ns, brr_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BRR_H */
