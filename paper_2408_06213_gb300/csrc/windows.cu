// windows.cu -- applying the swaps of a Fisher-Yates shuffle (Algorithm 1)
// by deterministic reservations over windows of consecutive steps, one CTA
// per array staged in shared memory.  Used by brr_shuffle_batched for the
// size ranges where it beats chain resolution (chains.cu): the arrays of the
// small class, and the larger ones that stage whole with a reservation table
// of at least 2,048 words, in 256-thread CTAs four per SM up to 8,016 4-byte
// elements, in 512-thread CTAs two per SM up to 17,744 and in 1024-thread
// CTAs up to 37,072; then, staging only the elements, up to 55,608.
//
// The steps p = n-1, n-2, ..., 1 are taken W at a time (W = the CTA's
// threads, one step each), in the sequential order of Algorithm 1.  A window
// is finished in rounds: every pending step reserves its two slots p and j_p
// by an atomic maximum of its priority (an earlier step in the sequential
// order, i.e. a larger p, has the higher priority) on the slots' reservation
// words, and commits -- exchanges the two elements -- when it holds both.
// A step that commits is the earliest pending step touching either of its
// slots, and the steps committing in one round touch disjoint slots, so the
// result is the sequential permutation.  Within a window of consecutive
// steps conflicts are rare (two steps with one target, or a step whose target
// is a later step's position), so most windows finish in a few rounds; the
// last windows, whose targets crowd into few slots, take more.  Steps with
// j_p = p exchange nothing and are left out.
//
// Reservation words carry a round counter above the priority: a word left by
// an earlier round is below every key of the current round, so nothing is
// cleared between rounds or windows.  The table has M words, slot x using
// word x mod M.  When M < n two slots can share a word; that only delays a
// step to a later round (a conflict that is not real) and never lets two
// steps that touch one slot commit together, and the pending step of highest
// priority always holds both its words, so every round commits a step.
//
// The array's swap targets are rolled first (Algorithm 4 batches, one thread
// per batch) into 16-bit words of shared memory, beside the elements and the
// table -- or, for the longest arrays, into the CTA's slot in global memory,
// which stays in L2 and is read once per window.
#include <algorithm>

#include "brr_common.cuh"
#include "internal.h"
#include "words.cuh"

namespace brr {

constexpr uint32_t kWinCap = 65536;         // 16-bit swap targets
constexpr uint32_t kWinPrioBits = 12;       // priorities 1 .. W <= 2048
constexpr int kWinSteps = 1;                // steps per thread in a window (two measured slower)
constexpr uint32_t kWinStageTable = 2048;   // a table of at least min(n, this) words (1024-thread class)

struct WinCtl {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
    int err;
    uint32_t item;
};

struct WinArgs {
    void *data;
    const uint64_t *offsets;
    const uint64_t *seeds;
    uint32_t n_arrays;
    uint64_t nk[BRR_SCHED_KMAX + 1];
    uint32_t k_max;
    uint32_t max_len;
    uint32_t *queue;        // the class's work counter
    const uint32_t *list;   // the class's arrays (null: every array, the others skipped)
    const uint32_t *count;  //   and how many
    uint16_t *jt_slots;     // targets in global memory: one slot of jt_slot elements per CTA
    uint32_t jt_slot;       //   (the class whose arrays stage only their elements)
    int *err;
};

struct WinClass {
    uint32_t lo, hi;    // arrays with lo < n <= hi
    uint32_t smem;      // dynamic shared memory per CTA
    uint32_t floor;     // smallest reservation table (words) an array may use
    uint32_t validate;  // record BRR_EINVAL for invalid arrays
};

__host__ __device__ __forceinline__ uint32_t win_pow2_floor(uint32_t x) {
    uint32_t p = 1;
    while (p <= x / 2) p <<= 1;
    return p;
}

__host__ __device__ __forceinline__ uint32_t win_pow2_ceil(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Shared memory of an array of n elements of eb bytes in `smem` bytes: the
// swap targets (none when they are kept in global memory), the elements,
// then the M reservation words.  `fits` when the table has at least min(n
// rounded up to a power of two, floor) words.
struct WinLayout {
    uint32_t jt_bytes, el_bytes, M;
    bool fits;
    __host__ __device__ WinLayout(uint32_t n, uint32_t eb, uint32_t smem, uint32_t floor = kWinStageTable,
                                  bool jt_global = false) {
        jt_bytes = jt_global ? 0u : (2 * n + 15) & ~15u;
        el_bytes = (n * eb + 15) & ~15u;
        const uint32_t want = win_pow2_ceil(n);
        const uint32_t rest = smem > jt_bytes + el_bytes ? smem - jt_bytes - el_bytes : 0u;
        const uint32_t f = rest >= 4 ? win_pow2_floor(rest / 4) : 0u;
        M = f < want ? f : want;
        fits = M >= 1 && M >= (want < floor ? want : floor);
    }
};

// The windows of one array on its elements A in shared memory, kSteps steps
// per thread (a window of W = kThreads * kSteps steps).  Returns false (the
// same in every thread) if a window needed more rounds than it has steps,
// which cannot happen.
template <typename T, int kThreads, int kSteps, bool kJtGlobal = false>
__device__ __forceinline__ bool win_apply(T *A, const uint16_t *jt, uint32_t *res, uint32_t mask, uint32_t n) {
    constexpr uint32_t W = (uint32_t)kThreads * kSteps;
    const uint32_t tid = threadIdx.x;
    uint32_t epoch = 0;
    for (int32_t top = (int32_t)n - 1; top >= 1; top -= (int32_t)W) {
        int32_t c[kSteps];
        uint32_t j[kSteps], rc[kSteps], rj[kSteps];
        bool pend[kSteps];
#pragma unroll
        for (int s = 0; s < kSteps; s++) {
            c[s] = top - (int32_t)(s * kThreads + tid);  // the thread's s-th step, earliest first
            j[s] = 0;
            pend[s] = false;
            if (c[s] >= 1) {
                j[s] = kJtGlobal ? __ldcg(jt + c[s]) : jt[c[s]];
                pend[s] = j[s] != (uint32_t)c[s];
            }
            rc[s] = (uint32_t)c[s] & mask;
            rj[s] = j[s] & mask;
        }
        for (uint32_t round = 0;; round++) {
            if (round > W) return false;
            epoch++;
#pragma unroll
            for (int s = 0; s < kSteps; s++) {
                if (pend[s]) {
                    const uint32_t key = (epoch << kWinPrioBits) | (W - (s * kThreads + tid));
                    atomicMax(&res[rc[s]], key);
                    atomicMax(&res[rj[s]], key);
                }
            }
            __syncthreads();
            bool any = false;
#pragma unroll
            for (int s = 0; s < kSteps; s++) {
                const uint32_t key = (epoch << kWinPrioBits) | (W - (s * kThreads + tid));
                if (pend[s] && res[rc[s]] == key && res[rj[s]] == key) {
                    const T x = A[c[s]];
                    A[c[s]] = A[j[s]];
                    A[j[s]] = x;
                    pend[s] = false;
                }
                any = any || pend[s];
            }
            if (!__syncthreads_or(any)) break;
        }
    }
    return true;
}

// kJtGlobal: the targets go to this CTA's slot in global memory (L2) and
// only the elements stage in shared memory, for arrays too long to stage
// both.
template <typename T, int kThreads, uint32_t SRC, bool kJtGlobal = false>
__global__ void __launch_bounds__(kThreads) win_cta_kernel(WinArgs a, WinClass cls) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ WinCtl ctl;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) ctl.err = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) ctl.item = atomicAdd(a.queue, 1u);
        __syncthreads();
        uint32_t s = ctl.item;
        if (a.list) {
            if (s >= *a.count) break;
            s = a.list[s];
        } else if (s >= a.n_arrays) {
            break;
        }
        const uint64_t o0 = a.offsets[s], o1 = a.offsets[s + 1];
        if (o1 < o0 || o1 - o0 > a.max_len) {
            if (cls.validate && tid == 0) ctl.err = BRR_EINVAL;
            continue;
        }
        const uint64_t len = o1 - o0;
        if (len < 2 || len <= cls.lo || len > cls.hi) continue;
        const uint32_t n = (uint32_t)len;
        const uint64_t seed = a.seeds[s];
        const WinLayout lay(n, (uint32_t)sizeof(T), cls.smem, cls.floor, kJtGlobal);
        if (tid == 0) {
            ctl.nseg = plan_segments(n, 1, a.nk, a.k_max, ctl.seg, kMaxSegs, &ctl.n_batches);
            if (ctl.nseg < 0 || !lay.fits) {  // (the host routes only arrays that fit)
                ctl.err = BRR_EINVAL;
                ctl.nseg = 0;
            }
        }
        T *g = static_cast<T *>(a.data) + o0;
        uint16_t *jt = kJtGlobal ? a.jt_slots + (size_t)blockIdx.x * a.jt_slot : reinterpret_cast<uint16_t *>(smem);
        T *As = reinterpret_cast<T *>(smem + lay.jt_bytes);
        uint32_t *res = reinterpret_cast<uint32_t *>(smem + lay.jt_bytes + lay.el_bytes);
        for (uint32_t x = tid; x < n; x += kThreads) As[x] = g[x];
        for (uint32_t x = tid; x < lay.M; x += kThreads) res[x] = 0;
        __syncthreads();
        if (ctl.nseg == 0) continue;
        roll_plan_range_src<SRC>(ctl.seg, ctl.nseg, 0, ctl.n_batches, seed, ctl.err,
                                 [&](uint32_t pos, uint32_t v) { jt[pos] = (uint16_t)v; });
        __syncthreads();
        const bool ok = win_apply<T, kThreads, kWinSteps, kJtGlobal>(As, jt, res, lay.M - 1, n);
        __syncthreads();
        for (uint32_t x = tid; x < n; x += kThreads) g[x] = As[x];
        if (!ok && tid == 0) ctl.err = BRR_ETIMEOUT;
    }
    __syncthreads();
    if (tid == 0 && ctl.err) record_error(a.err, ctl.err);
}

// ------------------------------------------------------------ launchers --
// Dynamic shared memory of a class: the large class (1024 threads, one CTA
// per SM) takes the whole opt-in amount, the middle one (512 threads) half of
// an SM and the quarter one (256 threads) a quarter, so that two or four CTAs
// overlap each other's barrier waits; the small one (128 threads) what its
// longest array needs with a full table.
constexpr uint32_t kWinMidFloor = 2048;  // the middle class accepts tables down to this size

static uint32_t win_limit(const brr_ctx *ctx) {
    return (uint32_t)(((size_t)ctx->max_smem_optin - sizeof(WinCtl) - 1024) & ~(size_t)15);
}

// Shared memory of one of `parts` CTAs that share an SM.
static uint32_t win_part_smem(const brr_ctx *ctx, uint32_t parts) {
    int per_sm = 0, reserved = 0;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device) != cudaSuccess) {
        cudaGetLastError();
        per_sm = (int)ctx->max_smem_optin;
        reserved = 1024;
    }
    const size_t part = ((size_t)per_sm - parts * (size_t)reserved) / parts;
    return (uint32_t)((part - sizeof(WinCtl) - 256) & ~(size_t)15);
}

static uint32_t win_mid_smem(const brr_ctx *ctx) { return win_part_smem(ctx, 2); }
static uint32_t win_quarter_smem(const brr_ctx *ctx) { return win_part_smem(ctx, 4); }

static uint32_t win_cap(uint32_t elem_bytes, uint32_t smem, uint32_t floor, bool jt_global = false) {
    uint32_t lo = 2, hi = kWinCap;  // the largest n that fits: fits is monotone in n
    if (WinLayout(hi, elem_bytes, smem, floor, jt_global).fits) return hi;
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (WinLayout(mid, elem_bytes, smem, floor, jt_global).fits) lo = mid;
        else hi = mid;
    }
    return lo;
}

uint32_t windows_stage_cap(const brr_ctx *ctx, uint32_t elem_bytes) {
    return win_cap(elem_bytes, win_limit(ctx), kWinStageTable);
}

uint32_t windows_mid_cap(const brr_ctx *ctx, uint32_t elem_bytes) {
    return win_cap(elem_bytes, win_mid_smem(ctx), kWinMidFloor);
}

uint32_t windows_quarter_cap(const brr_ctx *ctx, uint32_t elem_bytes) {
    return win_cap(elem_bytes, win_quarter_smem(ctx), kWinMidFloor);
}

uint32_t windows_xl_cap(const brr_ctx *ctx, uint32_t elem_bytes) {
    return win_cap(elem_bytes, win_limit(ctx), kWinStageTable, true);
}

uint32_t windows_xl_grid(const brr_ctx *ctx) { return (uint32_t)ctx->num_sms; }

template <typename T, int kThreads, uint32_t SRC, bool kJtGlobal = false>
static brr_status win_launch(brr_ctx *ctx, const WinArgs &a, uint32_t lo, uint32_t hi, bool validate,
                             cudaStream_t stream) {
    uint32_t smem = win_limit(ctx), floor = kWinStageTable;
    if (kThreads == 512) {
        smem = win_mid_smem(ctx);
        floor = kWinMidFloor;
    } else if (kThreads == 256) {
        smem = win_quarter_smem(ctx);
        floor = kWinMidFloor;
    } else if (kThreads < 256) {
        const uint32_t h = std::max(hi, 2u);
        smem = std::min(smem, ((2 * h + 15) & ~15u) + ((h * (uint32_t)sizeof(T) + 15) & ~15u) +
                                  4 * win_pow2_ceil(h));
    }
    const void *k = (const void *)win_cta_kernel<T, kThreads, SRC, kJtGlobal>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
    if (e != cudaSuccess || per_sm < 1) return BRR_ECUDA;
    uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)per_sm * ctx->num_sms, a.n_arrays);
    if (kJtGlobal) grid = std::min(grid, windows_xl_grid(ctx));  // one target slot per CTA
    win_cta_kernel<T, kThreads, SRC, kJtGlobal><<<grid, kThreads, smem, stream>>>(
        a, WinClass{lo, hi, smem, floor, validate ? 1u : 0u});
    return cuda_status(cudaGetLastError());
}

template <typename T, uint32_t SRC>
static brr_status win_range(brr_ctx *ctx, const WinArgs &a, uint32_t cls, uint32_t lo, uint32_t hi, bool validate,
                            cudaStream_t stream) {
    if (cls == 4) return win_launch<T, 1024, SRC, true>(ctx, a, lo, hi, validate, stream);
    if (cls == 2) return win_launch<T, 1024, SRC>(ctx, a, lo, hi, validate, stream);
    if (cls == 1) return win_launch<T, 512, SRC>(ctx, a, lo, hi, validate, stream);
    if (cls == 3) return win_launch<T, 256, SRC>(ctx, a, lo, hi, validate, stream);
    return win_launch<T, 128, SRC>(ctx, a, lo, hi, validate, stream);
}

brr_status launch_windows_range(brr_ctx *ctx, void *data, const uint64_t *offsets, uint32_t n_arrays,
                                uint32_t elem_bytes, const uint64_t *seeds, uint64_t max_len, const uint64_t *nk,
                                uint32_t k_max, uint32_t cls, uint32_t lo, uint32_t hi, uint32_t *queue,
                                const uint32_t *list, const uint32_t *count, bool validate, cudaStream_t stream,
                                uint32_t source, uint16_t *jt_slots) {
    hi = std::min(hi, kWinCap);
    if (hi <= lo) return BRR_OK;
    if (cls == 4 && !jt_slots) return BRR_EINVAL;
    WinArgs a = {};
    a.data = data;
    a.offsets = offsets;
    a.seeds = seeds;
    a.n_arrays = n_arrays;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = nk[k];
    a.k_max = k_max;
    a.max_len = (uint32_t)std::min<uint64_t>(max_len, 0xFFFFFFFFull);
    a.queue = queue;
    a.list = list;
    a.count = count;
    a.jt_slots = jt_slots;
    a.jt_slot = kWinCap;
    a.err = ctx->d_err;
    const bool eb4 = elem_bytes == 4;
    if (source == BRR_WORDS_CHACHA20)
        return eb4 ? win_range<uint32_t, BRR_WORDS_CHACHA20>(ctx, a, cls, lo, hi, validate, stream)
                   : win_range<uint64_t, BRR_WORDS_CHACHA20>(ctx, a, cls, lo, hi, validate, stream);
    if (source == BRR_WORDS_SPLITMIX32)
        return eb4 ? win_range<uint32_t, BRR_WORDS_SPLITMIX32>(ctx, a, cls, lo, hi, validate, stream)
                   : win_range<uint64_t, BRR_WORDS_SPLITMIX32>(ctx, a, cls, lo, hi, validate, stream);
    return eb4 ? win_range<uint32_t, BRR_WORDS_SPLITMIX64>(ctx, a, cls, lo, hi, validate, stream)
               : win_range<uint64_t, BRR_WORDS_SPLITMIX64>(ctx, a, cls, lo, hi, validate, stream);
}

}  // namespace brr
