// batched.cu -- many independent shuffles (Algorithm 1 with Algorithm 4
// batches, one seed per array) and many partial Fisher-Yates samples in one
// persistent launch each.
//
// A CTA takes one array (or one sample request) at a time from a device work
// counter and runs the whole method on it: plan, batched dice (Theorem 1
// chains, one thread per batch) and the deterministic-reservation rounds of
// shuffle.cu, separated by CTA barriers instead of grid barriers.  Arrays
// that fit are staged in shared memory (elements, reservation words and
// 16-bit swap indices); longer arrays are worked on in place with the
// reservation words and swap indices in a per-CTA slice of global scratch.
//
// Samples work on a compact slot space: the dense slots stop..n-1 of the
// identity array map to 0..D-1 and every swap target below `stop` gets the
// next free compact slot through an open-addressing hash table, so the n
// slots of the identity array are never materialised.
#include <algorithm>

#include "brr_common.cuh"
#include "internal.h"

namespace brr {

constexpr int kBatThreads = 512;
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

template <typename J> struct Done;
template <> struct Done<uint16_t> { static constexpr uint16_t v = 0xFFFFu; };
template <> struct Done<uint32_t> { static constexpr uint32_t v = 0xFFFFFFFFu; };

struct BatchCtl {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
    int err;
    uint32_t item;
    uint32_t hash_count;
};

// Rolls every batch of the CTA's current plan (in ctl) and stores the swap
// target of position i-1-m as map(a_m) into jt.
template <typename J, typename Map>
__device__ void cta_roll_plan(BatchCtl &ctl, uint64_t seed, J *jt, Map map) {
    for (uint64_t g = threadIdx.x; g < ctl.n_batches; g += blockDim.x) {
        int s = 0;
        while (s + 1 < ctl.nseg && ctl.seg[s + 1].g0 <= g) s++;
        const Seg sg = ctl.seg[s];
        const uint32_t k = sg.k;
        const uint32_t i = sg.i0 - (uint32_t)(g - sg.g0) * k;
        uint32_t a[BRR_SCHED_KMAX];
        uint32_t att = 0;
        uint64_t r = word(seed, g, 0);
#pragma unroll
        for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
            if (m < k) a[m] = chain_step(r, i - m);
        if (r < sg.u) {
            const uint64_t B = (uint64_t)falling(i, k);
            const uint64_t t = (0 - B) % B;
            while (r < t) {
                if (++att >= kMaxAttempts) { ctl.err = BRR_ERETRY; break; }
                r = word(seed, g, att);
#pragma unroll
                for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
                    if (m < k) a[m] = chain_step(r, i - m);
            }
        }
#pragma unroll
        for (uint32_t m = 0; m < BRR_SCHED_KMAX; m++)
            if (m < k) map(i - 1 - m, a[m]);
    }
}

// Deterministic-reservation rounds on positions p_lo..P-1 of one CTA-local
// problem: position p swaps slots p and jt[p] (jt[p] == Done: no step) with
// priority p + 1 (later positions come first in the sequential order).  res
// must be zero on entry and is zero again on exit.  The same code runs on
// shared memory and on global scratch (CTA barriers order both).
template <typename T, typename J>
__device__ void cta_rounds(BatchCtl &ctl, T *A, uint32_t *res, J *jt, uint32_t p_lo, uint32_t P) {
    // every round commits the earliest pending swap, so P - p_lo + 1 rounds
    // always suffice; more means corrupted state, reported instead of looping
    for (uint32_t round = 0;; round++) {
        if (round > P - p_lo + 1) {
            if (threadIdx.x == 0) ctl.err = BRR_ETIMEOUT;
            break;
        }
        for (uint32_t p = p_lo + threadIdx.x; p < P; p += blockDim.x) {
            const J jp = jt[p];
            if (jp == Done<J>::v) continue;
            atomicMax(&res[p], p + 1);
            if ((uint32_t)jp != p) atomicMax(&res[jp], p + 1);
        }
        __syncthreads();
        bool pend = false;
        for (uint32_t p = p_lo + threadIdx.x; p < P; p += blockDim.x) {
            const J jp = jt[p];
            if (jp == Done<J>::v) continue;
            if (res[p] == p + 1 && res[jp] == p + 1) {
                if ((uint32_t)jp != p) {
                    const T x = A[p];
                    A[p] = A[jp];
                    A[jp] = x;
                }
                res[p] = 0;
                res[jp] = 0;
                jt[p] = Done<J>::v;
            } else {
                pend = true;
            }
        }
        if (__syncthreads_or(pend) == 0) break;
    }
}

// ------------------------------------------------------------- shuffles --
struct BatchedArgs {
    void *data;
    const uint64_t *offsets;
    const uint64_t *seeds;
    uint32_t n_arrays;
    uint64_t nk[BRR_SCHED_KMAX + 1];
    uint32_t k_max;
    uint32_t smem_cap;    // longest array staged in shared memory
    uint32_t max_len;
    uint32_t n_slots;     // CTAs 0..n_slots-1 own a global scratch slice
    uint32_t *slot_res;   // [n_slots][max_len]
    uint32_t *slot_j;     // [n_slots][max_len]
    uint32_t *queue;      // [2]: next small array, next big array
    int *err;
};

template <typename T>
__device__ void shuffle_in_smem(BatchCtl &ctl, const BatchedArgs &a, T *g, uint32_t n,
                                uint64_t seed, unsigned char *smem) {
    T *As = reinterpret_cast<T *>(smem);
    uint32_t *res = reinterpret_cast<uint32_t *>(smem + (((size_t)n * sizeof(T) + 15) & ~(size_t)15));
    uint16_t *jt = reinterpret_cast<uint16_t *>(res + n);
    for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) {
        As[x] = g[x];
        res[x] = 0;
    }
    if (threadIdx.x == 0) jt[0] = Done<uint16_t>::v;
    __syncthreads();
    cta_roll_plan<uint16_t>(ctl, seed, jt, [&](uint32_t pos, uint32_t v) { jt[pos] = (uint16_t)v; });
    __syncthreads();
    cta_rounds<T, uint16_t>(ctl, As, res, jt, 1, n);
    for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) g[x] = As[x];
}

template <typename T>
__device__ void shuffle_in_global(BatchCtl &ctl, const BatchedArgs &a, T *g, uint32_t n,
                                  uint64_t seed, uint32_t slot) {
    uint32_t *res = a.slot_res + (size_t)slot * a.max_len;
    uint32_t *jt = a.slot_j + (size_t)slot * a.max_len;
    for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) res[x] = 0;
    if (threadIdx.x == 0) jt[0] = Done<uint32_t>::v;
    __syncthreads();
    cta_roll_plan<uint32_t>(ctl, seed, jt, [&](uint32_t pos, uint32_t v) { jt[pos] = v; });
    __syncthreads();
    cta_rounds<T, uint32_t>(ctl, g, res, jt, 1, n);
}

template <typename T>
__global__ void __launch_bounds__(kBatThreads) shuffle_batched_kernel(BatchedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BatchCtl ctl;
    if (threadIdx.x == 0) ctl.err = 0;
    // CTAs that own a scratch slice first drain the queue of long arrays.
    for (int phase = (blockIdx.x < a.n_slots) ? 1 : 0; phase >= 0; phase--) {
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) ctl.item = atomicAdd(&a.queue[phase], 1u);
            __syncthreads();
            const uint32_t s = ctl.item;
            if (s >= a.n_arrays) break;
            const uint64_t o0 = a.offsets[s], o1 = a.offsets[s + 1];
            if (o1 < o0 || o1 - o0 > a.max_len) {
                if (phase == 0 && threadIdx.x == 0) ctl.err = BRR_EINVAL;
                continue;
            }
            const uint32_t n = (uint32_t)(o1 - o0);
            const bool big = n > a.smem_cap;
            if (big != (phase == 1) || n < 2) continue;
            if (threadIdx.x == 0) {
                ctl.nseg = plan_segments(n, 1, a.nk, a.k_max, ctl.seg, kMaxSegs, &ctl.n_batches);
                if (ctl.nseg < 0) { ctl.err = BRR_EINVAL; ctl.n_batches = 0; ctl.nseg = 0; }
            }
            __syncthreads();
            if (ctl.nseg == 0) continue;
            T *g = static_cast<T *>(a.data) + o0;
            if (big) shuffle_in_global<T>(ctl, a, g, n, a.seeds[s], blockIdx.x);
            else shuffle_in_smem<T>(ctl, a, g, n, a.seeds[s], smem);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && ctl.err) record_error(a.err, ctl.err);
}

static size_t smem_bytes_for(uint32_t cap, uint32_t eb) {
    return (((size_t)cap * eb + 15) & ~(size_t)15) + (size_t)cap * 4 + (size_t)cap * 2 + 16;
}

brr_status launch_shuffle_batched(brr_ctx *ctx, void *data, const uint64_t *offsets,
                                  uint32_t n_arrays, uint32_t elem_bytes, const uint64_t *seeds,
                                  uint64_t max_len, const brr_schedule *sched,
                                  cudaStream_t stream) {
    BatchedArgs a;
    a.data = data;
    a.offsets = offsets;
    a.seeds = seeds;
    a.n_arrays = n_arrays;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = sched->n_k[k];
    a.k_max = sched->k_max;
    a.max_len = (uint32_t)max_len;
    a.err = ctx->d_err;
    // shared memory: the largest staging area that still lets the CTA run
    const size_t smem_limit = (size_t)ctx->max_smem_optin - sizeof(BatchCtl) - 1024;
    const uint32_t per_elem = elem_bytes + 4 + 2;
    uint32_t cap = (uint32_t)std::min<uint64_t>((smem_limit - 32) / per_elem, 65534);
    if ((uint64_t)cap > max_len) cap = (uint32_t)max_len;
    a.smem_cap = cap;
    const size_t smem = smem_bytes_for(std::max<uint32_t>(cap, 1), elem_bytes);
    const void *kern = elem_bytes == 4 ? (const void *)shuffle_batched_kernel<uint32_t>
                                       : (const void *)shuffle_batched_kernel<uint64_t>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatThreads, smem);
    if (per_sm < 1) return BRR_ECUDA;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)per_sm * ctx->num_sms, n_arrays);
    // scratch slices for arrays longer than the staging capacity
    uint32_t n_slots = 0;
    size_t slot_bytes = 0;
    if (max_len > cap) {
        slot_bytes = (size_t)max_len * 8;
        const size_t budget = (size_t)1 << 30;
        n_slots = (uint32_t)std::max<size_t>(1, std::min<size_t>(grid, budget / slot_bytes));
    }
    const size_t need = 256 + (size_t)n_slots * slot_bytes;
    brr_status st = ensure_scratch(ctx, need);
    if (st != BRR_OK) return st;
    char *base = static_cast<char *>(ctx->scratch);
    a.queue = reinterpret_cast<uint32_t *>(base);
    a.n_slots = n_slots;
    a.slot_res = reinterpret_cast<uint32_t *>(base + 256);
    a.slot_j = a.slot_res + (size_t)n_slots * max_len;
    e = cudaMemsetAsync(a.queue, 0, 2 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (elem_bytes == 4)
        shuffle_batched_kernel<uint32_t><<<grid, kBatThreads, smem, stream>>>(a);
    else
        shuffle_batched_kernel<uint64_t><<<grid, kBatThreads, smem, stream>>>(a);
    return cuda_status(cudaGetLastError());
}

// -------------------------------------------------------------- samples --
struct SampleArgs {
    const uint64_t *n;
    const uint32_t *m;
    const uint64_t *seeds;
    const uint64_t *out_off;
    uint32_t n_req;
    uint64_t single_n;  // used when n == nullptr (one request)
    uint32_t single_m;
    uint64_t single_seed;
    uint64_t nk[BRR_SCHED_KMAX + 1];
    uint32_t k_max;
    uint32_t max_m;
    uint32_t smem_cap_m;  // largest m whose work arrays fit shared memory
    uint32_t *out;
    uint32_t *queue;
    uint32_t n_slots;
    size_t slot_words;    // uint32 words per scratch slice
    uint32_t *slots;
    int *err;
};

// Work arrays of one sample with D dense slots: values and reservations for
// up to 2D compact slots, compact swap targets for D positions, and a hash
// table of H (power of two, >= 2D) keys and compact indices.
__host__ __device__ inline uint32_t sample_hash_size(uint32_t D) {
    uint32_t H = 16;
    while (H < 2 * D) H <<= 1;
    return H;
}
__host__ __device__ inline size_t sample_words(uint32_t D) {
    return (size_t)2 * D * 2 + D + 2 * (size_t)sample_hash_size(D) + 8;
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t key, uint32_t mask) {
    return (uint32_t)(((uint64_t)key * 0x9E3779B97F4A7C15ull) >> 32) & mask;
}

// Inserts key s (a swap target below `stop`) into the open-addressing table
// (keys only; compact indices are assigned afterwards).  The table holds at
// least twice as many entries as there can be keys, so probing ends.
__device__ void hash_insert(uint32_t *keys, uint32_t mask, uint32_t s) {
    uint32_t h = hash_slot(s, mask);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const uint32_t prev = atomicCAS(&keys[h], kEmptyKey, s);
        if (prev == kEmptyKey || prev == s) return;
        h = (h + 1) & mask;
    }
}

__device__ uint32_t hash_find(const uint32_t *keys, const uint32_t *vals, uint32_t mask, uint32_t s) {
    uint32_t h = hash_slot(s, mask);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const uint32_t k = keys[h];
        if (k == s) return vals[h];
        if (k == kEmptyKey) return kEmptyKey;
        h = (h + 1) & mask;
    }
    return kEmptyKey;
}

__device__ void sample_one(BatchCtl &ctl, const SampleArgs &a, uint32_t n, uint32_t m,
                           uint64_t seed, uint32_t *out, uint32_t *w) {
    const uint32_t stop = (n - m) > 1 ? (n - m) : 1;
    const uint32_t D = n - stop;              // steps = dense slots
    const uint32_t H = sample_hash_size(D);
    uint32_t *Ac = w;                         // [2D] values
    uint32_t *res = Ac + 2 * D;               // [2D] reservations
    uint32_t *jc = res + 2 * D;               // [D] compact targets (Done: none)
    uint32_t *keys = jc + D;                  // [H]
    uint32_t *vals = keys + H;                // [H]
    for (uint32_t x = threadIdx.x; x < 2 * D; x += blockDim.x) {
        Ac[x] = x < D ? stop + x : 0;
        res[x] = 0;
    }
    for (uint32_t x = threadIdx.x; x < H; x += blockDim.x) {
        keys[x] = kEmptyKey;
        vals[x] = kEmptyKey;
    }
    if (threadIdx.x == 0) ctl.hash_count = 0;
    __syncthreads();
    // 1. roll the plan; position p of the identity array is compact slot
    //    p - stop, and targets below stop are collected in the hash table
    cta_roll_plan<uint32_t>(ctl, seed, jc, [&](uint32_t pos, uint32_t v) {
        jc[pos - stop] = v;
        if (v < stop) hash_insert(keys, H - 1, v);
    });
    __syncthreads();
    // 2. number the collected targets: compact slots D, D+1, ...
    for (uint32_t h = threadIdx.x; h < H; h += blockDim.x) {
        const uint32_t key = keys[h];
        if (key != kEmptyKey) {
            const uint32_t idx = D + atomicAdd(&ctl.hash_count, 1u);
            vals[h] = idx;
            Ac[idx] = key;
        }
    }
    __syncthreads();
    // 3. swap targets in compact coordinates
    for (uint32_t c = threadIdx.x; c < D; c += blockDim.x) {
        const uint32_t v = jc[c];
        jc[c] = v >= stop ? v - stop : hash_find(keys, vals, H - 1, v);
    }
    __syncthreads();
    cta_rounds<uint32_t, uint32_t>(ctl, Ac, res, jc, 0, D);
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < m; q += blockDim.x) {
        uint32_t v;
        if (q < D) {
            v = Ac[D - 1 - q];
        } else {  // m == n: the value left in slot 0
            const uint32_t c = hash_find(keys, vals, H - 1, 0);
            v = c == kEmptyKey ? 0 : Ac[c];
        }
        out[q] = v;
    }
}

__global__ void __launch_bounds__(kBatThreads) sample_kernel(SampleArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BatchCtl ctl;
    if (threadIdx.x == 0) ctl.err = 0;
    for (int phase = (blockIdx.x < a.n_slots) ? 1 : 0; phase >= 0; phase--) {
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) ctl.item = atomicAdd(&a.queue[phase], 1u);
            __syncthreads();
            const uint32_t r = ctl.item;
            if (r >= a.n_req) break;
            const uint64_t n = a.n ? a.n[r] : a.single_n;
            const uint32_t m = a.n ? a.m[r] : a.single_m;
            const uint64_t seed = a.n ? a.seeds[r] : a.single_seed;
            const uint64_t oo = a.n ? a.out_off[r] : 0;
            if (n > 0xFFFFFFFFull || m > n || m > a.max_m) {
                if (phase == 0 && threadIdx.x == 0) ctl.err = BRR_EINVAL;
                continue;
            }
            if (m == 0) continue;
            const bool big = m > a.smem_cap_m;
            if (big != (phase == 1)) continue;
            const uint32_t stop = (uint32_t)((n - m) > 1 ? (n - m) : 1);
            if (threadIdx.x == 0) {
                ctl.nseg = plan_segments(n, stop, a.nk, a.k_max, ctl.seg, kMaxSegs, &ctl.n_batches);
                if (ctl.nseg < 0) { ctl.err = BRR_EINVAL; ctl.nseg = 0; ctl.n_batches = 0; }
            }
            __syncthreads();
            uint32_t *w = big ? a.slots + (size_t)blockIdx.x * a.slot_words
                              : reinterpret_cast<uint32_t *>(smem);
            sample_one(ctl, a, (uint32_t)n, m, seed, a.out + oo, w);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && ctl.err) record_error(a.err, ctl.err);
}

brr_status launch_sample_batched(brr_ctx *ctx, const uint64_t *n, const uint32_t *m,
                                 const uint64_t *seeds, const uint64_t *out_off, uint32_t n_req,
                                 uint32_t max_m, const brr_schedule *sched, uint32_t *out,
                                 cudaStream_t stream, const uint64_t *host_n_single,
                                 uint32_t host_m_single, uint64_t host_seed_single) {
    SampleArgs a;
    a.n = n;
    a.m = m;
    a.seeds = seeds;
    a.out_off = out_off;
    a.n_req = n_req;
    a.single_n = host_n_single ? *host_n_single : 0;
    a.single_m = host_m_single;
    a.single_seed = host_seed_single;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = sched->n_k[k];
    a.k_max = sched->k_max;
    a.max_m = max_m;
    a.out = out;
    a.err = ctx->d_err;
    const size_t smem_limit = (size_t)ctx->max_smem_optin - sizeof(BatchCtl) - 1024;
    uint32_t cap = 16;
    while (cap * 2 <= max_m && sample_words(cap * 2) * 4 <= smem_limit) cap *= 2;
    while (cap + 16 <= max_m && sample_words(cap + 16) * 4 <= smem_limit) cap += 16;
    if (cap > max_m) cap = max_m;
    a.smem_cap_m = cap;
    const size_t smem = sample_words(cap) * 4;
    const void *kern = (const void *)sample_kernel;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatThreads, smem);
    if (per_sm < 1) return BRR_ECUDA;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)per_sm * ctx->num_sms, n_req);
    a.n_slots = 0;
    a.slot_words = 0;
    if (max_m > cap) {
        a.slot_words = (sample_words(max_m) + 63) & ~(size_t)63;
        const size_t budget = (size_t)1 << 30;
        a.n_slots = (uint32_t)std::max<size_t>(1, std::min<size_t>(grid, budget / (a.slot_words * 4)));
    }
    brr_status st = ensure_scratch(ctx, 256 + (size_t)a.n_slots * a.slot_words * 4);
    if (st != BRR_OK) return st;
    char *base = static_cast<char *>(ctx->scratch);
    a.queue = reinterpret_cast<uint32_t *>(base);
    a.slots = reinterpret_cast<uint32_t *>(base + 256);
    e = cudaMemsetAsync(a.queue, 0, 2 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    sample_kernel<<<grid, kBatThreads, smem, stream>>>(a);
    return cuda_status(cudaGetLastError());
}

}  // namespace brr
