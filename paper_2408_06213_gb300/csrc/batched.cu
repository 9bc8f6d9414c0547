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

#include <cooperative_groups.h>

#include "brr_common.cuh"
#include "internal.h"

namespace brr {

constexpr int kBatThreads = 512;
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

template <typename J> struct Done;
template <> struct Done<uint16_t> { static constexpr uint16_t v = 0xFFFFu; };
template <> struct Done<uint32_t> { static constexpr uint32_t v = 0xFFFFFFFFu; };

constexpr uint32_t kTailCap = 256;  // pending swaps finished sequentially

struct BatchCtl {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
    int err;
    uint32_t item;
    uint32_t hash_count;
    uint32_t pending[2];      // pending positions, by round parity
    uint32_t list[kTailCap];
};

template <typename J, typename Map>
__device__ void cta_roll_plan(BatchCtl &ctl, uint64_t seed, J *jt, Map map) {
    roll_plan_range(ctl.seg, ctl.nseg, 0, ctl.n_batches, seed, ctl.err, map);
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

// Bitmap-driven reservation rounds shared by the one-CTA and the cluster
// shuffles.  The pending positions of the CTA's own chunk are a bitmap (bit
// pl of bm = global position lo + pl).  A warp takes bitmap words warp,
// warp + nw, ... in groups of kU, so that the shared (or distributed shared)
// loads of kU words overlap: first every load a group needs (words, swap
// targets, the two reservation words), then the element loads of the swaps
// that commit, then all stores -- a few memory round trips per group rather
// than a few per position.  Words with nothing pending cost one load.
// slot(j) resolves global position j to its reservation word and element.
constexpr int kU = 4;

template <typename T>
struct SlotRef {
    uint32_t *res;
    T *a;
};

template <typename T, typename J, typename Slot>
__device__ __forceinline__ void reserve_pass(const uint32_t *bm, uint32_t nwords, const J *jt,
                                             uint32_t *res, uint32_t lo, Slot slot) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t w0 = warp; w0 < nwords; w0 += nw * kU) {
        uint32_t bits[kU], jp[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t w = w0 + u * nw;
            bits[u] = w < nwords ? bm[w] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kU; u++)
            jp[u] = ((bits[u] >> lane) & 1u) ? jt[32 * (w0 + u * nw) + lane] : 0u;
#pragma unroll
        for (int u = 0; u < kU; u++) {
            if ((bits[u] >> lane) & 1u) {
                const uint32_t pl = 32 * (w0 + u * nw) + lane, p = lo + pl;
                atomicMax(&res[pl], p + 1);
                if (jp[u] != p) atomicMax(slot(jp[u]).res, p + 1);
            }
        }
    }
}

// Returns how many positions of this warp's words are still pending (the
// same value in every lane).
template <typename T, typename J, typename Slot>
__device__ __forceinline__ uint32_t commit_pass(uint32_t *bm, uint32_t nwords, const J *jt, T *A,
                                                uint32_t *res, uint32_t lo, Slot slot) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t pend = 0;
    for (uint32_t w0 = warp; w0 < nwords; w0 += nw * kU) {
        uint32_t bits[kU];
        uint32_t any = 0;
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t w = w0 + u * nw;
            bits[u] = w < nwords ? bm[w] : 0u;
            any |= bits[u];
        }
        if (any == 0) continue;  // the same words for the whole warp
        bool ok[kU];
        uint32_t jp[kU];
        SlotRef<T> sj[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const bool mine = (bits[u] >> lane) & 1u;
            const uint32_t pl = mine ? 32 * (w0 + u * nw) + lane : 0u;  // in range when used
            jp[u] = mine ? jt[pl] : 0u;
            sj[u] = slot(jp[u]);
            ok[u] = mine && res[pl] == lo + pl + 1 && *sj[u].res == lo + pl + 1;
        }
        T va[kU], vb[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t pl = 32 * (w0 + u * nw) + lane;
            if (ok[u] && jp[u] != lo + pl) {
                va[u] = A[pl];
                vb[u] = *sj[u].a;
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t pl = 32 * (w0 + u * nw) + lane;
            if (ok[u]) {
                if (jp[u] != lo + pl) {
                    A[pl] = vb[u];
                    *sj[u].a = va[u];
                }
                res[pl] = 0;
                *sj[u].res = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t w = w0 + u * nw;
            const uint32_t nbits = __ballot_sync(0xffffffffu, ((bits[u] >> lane) & 1u) && !ok[u]);
            if (lane == 0 && w < nwords) bm[w] = nbits;
            pend += __popc(nbits);
        }
    }
    return pend;
}

// When few swaps are left pending, finishing them one window at a time is
// cheaper than more rounds: warp 0 lists the pending positions in decreasing
// order (the sequential order of Algorithm 1) and applies them 32 at a time.
// In a window, swap i must follow every earlier swap h that touches one of
// its slots: the same target (j_h == j_i) or h targeting i's own position
// (j_h == p_i) -- an earlier position is never i's target, as j_i <= p_i <
// p_h.  Ready swaps are applied in waves until the window is done.  The
// swaps already committed are closed under earlier conflicts, so applying the
// rest in order gives the sequential result.
constexpr uint32_t kTail = kTailCap;

template <typename T, typename WordAt, typename JAt, typename Slot>
__device__ void finish_pending(uint32_t nwords_total, uint32_t *list, WordAt word_at, JAt jt_at,
                               Slot slot) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t nl = 0;
    for (int32_t top = (int32_t)nwords_total - 1; top >= 0; top -= 32) {
        const int32_t w = top - (int32_t)lane;
        uint32_t bits = w >= 0 ? word_at((uint32_t)w) : 0u;
        const uint32_t cnt = __popc(bits);
        uint32_t pre = cnt;  // inclusive scan, lane 0 first (highest word)
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, pre, d);
            if ((int)lane >= d) pre += t;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, pre, 31);
        uint32_t pos = nl + pre - cnt;
        while (bits) {
            const uint32_t b = 31 - __clz(bits);
            if (pos < kTail) list[pos] = 32u * (uint32_t)w + b;
            pos++;
            bits &= ~(1u << b);
        }
        nl += total;
    }
    __syncwarp();
    if (nl > kTail) nl = kTail;  // callers only come here with at most kTail pending
    for (uint32_t base = 0; base < nl; base += 32) {
        const uint32_t i = base + lane;
        const bool act = i < nl;
        const uint32_t p = act ? list[i] : 0u;
        const uint32_t j = act ? (uint32_t)jt_at(p) : 0u;
        uint32_t deps = 0;
        for (uint32_t h = 0; h < 32; h++) {
            const uint32_t jh = __shfl_sync(0xffffffffu, j, h);
            if (h < lane && (jh == j || jh == p)) deps |= 1u << h;
        }
        uint32_t done = ~__ballot_sync(0xffffffffu, act);
        for (uint32_t wave = 0; wave < 32 && done != 0xffffffffu; wave++) {
            const bool ready = act && !((done >> lane) & 1u) && (deps & ~done) == 0;
            if (ready && j != p) {
                const SlotRef<T> sp = slot(p), sj = slot(j);
                const T x = *sp.a;
                *sp.a = *sj.a;
                *sj.a = x;
            }
            __syncwarp();
            done |= __ballot_sync(0xffffffffu, ready);
        }
    }
}

// Rounds for a shuffle worked on by one CTA: staged in its shared memory
// (J = uint16_t), or in place in global memory with the reservation words,
// swap indices and bitmap in a scratch slice (J = uint32_t), where the
// slice and the array stay resident in L2 while the CTA works on them.
template <typename T, typename J>
__device__ void cta_rounds_bitmap(BatchCtl &ctl, T *A, uint32_t *res, const J *jt,
                                  uint32_t *bm, uint32_t n) {
    const uint32_t nwords = (n + 31) / 32;
    auto slot = [&](uint32_t j) { return SlotRef<T>{res + j, A + j}; };
    for (uint32_t round = 0;; round++) {
        if (round > n + 1) {  // cannot happen: every round commits a swap
            if (threadIdx.x == 0) ctl.err = BRR_ETIMEOUT;
            break;
        }
        // pending[round & 1] is zero here: it was cleared after the first
        // barrier of the previous round, when every read of it was over
        if (round == 0 && threadIdx.x == 0) ctl.pending[0] = 0;
        reserve_pass<T, J>(bm, nwords, jt, res, 0, slot);
        __syncthreads();
        if (threadIdx.x == 0) ctl.pending[(round + 1) & 1u] = 0;
        const uint32_t pend = commit_pass<T, J>(bm, nwords, jt, A, res, 0, slot);
        if ((threadIdx.x & 31u) == 0 && pend) atomicAdd(&ctl.pending[round & 1u], pend);
        __syncthreads();
        const uint32_t left = ctl.pending[round & 1u];
        if (left == 0) break;
        if (left <= kTail) {
            if (threadIdx.x < 32)
                finish_pending<T>(nwords, ctl.list, [&](uint32_t w) { return bm[w]; },
                                  [&](uint32_t p) { return jt[p]; }, slot);
            __syncthreads();
            break;
        }
    }
}

// Pending bitmap word w for positions 1..n-1 of a shuffle (position 0 never
// swaps).
__device__ __forceinline__ uint32_t initial_pending_word(uint32_t w, uint32_t lo, uint32_t n) {
    const uint32_t first = lo + 32 * w;  // global position of bit 0
    uint32_t bits = 0xffffffffu;
    if (first + 32 > n) bits = first >= n ? 0u : (0xffffffffu >> (first + 32 - n));
    if (first == 0) bits &= ~1u;
    return bits;
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
    uint32_t *slot_res;   // [n_slots][slot_words]: reservations, swap indices, bitmap
    size_t slot_words;
    uint32_t *queue;      // [3]: next small array, next long array, next cluster array
    uint32_t cluster_cap; // arrays with smem_cap < n <= cluster_cap go to the cluster kernel
    uint32_t use_cluster; //   (when use_cluster is set; otherwise to the long kernel)
    uint32_t long_bm_smem;// the long kernel keeps its pending bitmap in shared memory
    // single-array form (offsets == nullptr): one shuffle of n elements
    uint32_t single_n;
    uint64_t single_seed;
    uint32_t *j_out;      // optional swap indices of the single array
    int *err;
};

template <typename T>
__device__ void shuffle_in_smem(BatchCtl &ctl, const BatchedArgs &a, T *g, uint32_t n,
                                uint64_t seed, unsigned char *smem) {
    T *As = reinterpret_cast<T *>(smem);
    uint32_t *res = reinterpret_cast<uint32_t *>(smem + (((size_t)n * sizeof(T) + 15) & ~(size_t)15));
    uint16_t *jt = reinterpret_cast<uint16_t *>(res + n);
    uint32_t *bm = reinterpret_cast<uint32_t *>(jt + ((n + 1) & ~1u));
    for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) {
        As[x] = g[x];
        res[x] = 0;
    }
    for (uint32_t w = threadIdx.x; w < (n + 31) / 32; w += blockDim.x) bm[w] = initial_pending_word(w, 0, n);
    __syncthreads();
    cta_roll_plan<uint16_t>(ctl, seed, jt, [&](uint32_t pos, uint32_t v) { jt[pos] = (uint16_t)v; });
    __syncthreads();
    if (a.j_out)
        for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) a.j_out[x] = x == 0 ? 0u : jt[x];
    cta_rounds_bitmap<T, uint16_t>(ctl, As, res, jt, bm, n);
    for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) g[x] = As[x];
}

template <typename T>
__device__ void shuffle_in_global(BatchCtl &ctl, const BatchedArgs &a, T *g, uint32_t n,
                                  uint64_t seed, uint32_t slot) {
    uint32_t *res = a.slot_res + (size_t)slot * a.slot_words;
    uint32_t *jt = res + a.max_len;
    // the pending bitmap lives in shared memory when it fits (scanned every round)
    extern __shared__ __align__(16) unsigned char lsmem[];
    uint32_t *bm = a.long_bm_smem ? reinterpret_cast<uint32_t *>(lsmem) : jt + a.max_len;
    for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) res[x] = 0;
    for (uint32_t w = threadIdx.x; w < (n + 31) / 32; w += blockDim.x) bm[w] = initial_pending_word(w, 0, n);
    __syncthreads();
    cta_roll_plan<uint32_t>(ctl, seed, jt, [&](uint32_t pos, uint32_t v) { jt[pos] = v; });
    __syncthreads();
    if (a.j_out)
        for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) a.j_out[x] = x == 0 ? 0u : jt[x];
    cta_rounds_bitmap<T, uint32_t>(ctl, g, res, jt, bm, n);
}

// Arrays up to the shared-memory capacity of one CTA, one CTA per array at a
// time; also validates every array (lengths above max_len are reported).
template <typename T>
__global__ void __launch_bounds__(kBatThreads) shuffle_batched_kernel(BatchedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BatchCtl ctl;
    if (threadIdx.x == 0) ctl.err = 0;
    const uint32_t n_items = a.offsets ? a.n_arrays : 1u;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) ctl.item = atomicAdd(&a.queue[0], 1u);
        __syncthreads();
        const uint32_t s = ctl.item;
        if (s >= n_items) break;
        uint64_t o0 = 0, o1 = a.single_n, seed = a.single_seed;
        if (a.offsets) {
            o0 = a.offsets[s];
            o1 = a.offsets[s + 1];
            seed = a.seeds[s];
        }
        if (o1 < o0 || o1 - o0 > a.max_len) {
            if (threadIdx.x == 0) ctl.err = BRR_EINVAL;
            continue;
        }
        const uint32_t n = (uint32_t)(o1 - o0);
        if (n > a.smem_cap || n < 2) continue;  // longer arrays: the other kernels
        if (threadIdx.x == 0) {
            ctl.nseg = plan_segments(n, 1, a.nk, a.k_max, ctl.seg, kMaxSegs, &ctl.n_batches);
            if (ctl.nseg < 0) { ctl.err = BRR_EINVAL; ctl.n_batches = 0; ctl.nseg = 0; }
        }
        __syncthreads();
        if (ctl.nseg == 0) continue;
        shuffle_in_smem<T>(ctl, a, static_cast<T *>(a.data) + o0, n, seed, smem);
    }
    __syncthreads();
    if (threadIdx.x == 0 && ctl.err) record_error(a.err, ctl.err);
}

// Arrays longer than one CTA's shared memory: one CTA per array, in place,
// with scratch slice blockIdx.x.  Little shared memory, so several CTAs share
// an SM and hide each other's L2 latency.
constexpr int kLongThreads = 256;
constexpr size_t kLongBitmapSmem = 32768;  // bitmap in shared memory up to 2^18 positions

template <typename T>
__global__ void __launch_bounds__(kLongThreads) shuffle_long_kernel(BatchedArgs a) {
    __shared__ BatchCtl ctl;
    if (threadIdx.x == 0) ctl.err = 0;
    const uint32_t n_items = a.offsets ? a.n_arrays : 1u;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) ctl.item = atomicAdd(&a.queue[1], 1u);
        __syncthreads();
        const uint32_t s = ctl.item;
        if (s >= n_items) break;
        uint64_t o0 = 0, o1 = a.single_n, seed = a.single_seed;
        if (a.offsets) {
            o0 = a.offsets[s];
            o1 = a.offsets[s + 1];
            seed = a.seeds[s];
        }
        if (o1 < o0 || o1 - o0 > a.max_len) continue;  // reported by the short kernel
        const uint32_t n = (uint32_t)(o1 - o0);
        if (n <= a.smem_cap || (a.use_cluster && n <= a.cluster_cap)) continue;
        if (threadIdx.x == 0) {
            ctl.nseg = plan_segments(n, 1, a.nk, a.k_max, ctl.seg, kMaxSegs, &ctl.n_batches);
            if (ctl.nseg < 0) { ctl.err = BRR_EINVAL; ctl.n_batches = 0; ctl.nseg = 0; }
        }
        __syncthreads();
        if (ctl.nseg == 0) continue;
        shuffle_in_global<T>(ctl, a, static_cast<T *>(a.data) + o0, n, seed, blockIdx.x);
    }
    __syncthreads();
    if (threadIdx.x == 0 && ctl.err) record_error(a.err, ctl.err);
}

static size_t smem_bytes_for(uint32_t cap, uint32_t eb) {
    return (((size_t)cap * eb + 15) & ~(size_t)15) + (size_t)cap * 4 + (size_t)(cap + 1) * 2 +
           (size_t)(cap + 31) / 32 * 4 + 16;
}

// ------------------------------------------------------ cluster shuffles --
// Arrays too long for one CTA's shared memory but at most kClSize *
// kClChunkCap elements are shuffled by a thread-block cluster: CTA r of the
// cluster holds positions [r*chunk, (r+1)*chunk) -- elements, reservation
// words, 16-bit swap indices and the pending bitmap -- in its shared memory,
// and reaches the other CTAs' slots through distributed shared memory
// (loads, stores and atomics on addresses from map_shared_rank).  Rounds are
// separated by cluster barriers; a round ends the shuffle when no CTA has a
// pending position left (counts added into CTA 0's shared memory); the last
// few pending swaps are finished in order by one warp.
constexpr int kClSize = 8;
constexpr uint32_t kClChunkCap = 8192;
constexpr uint32_t kClusterCap = kClSize * kClChunkCap;  // 65,536

struct ClusterCtl {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
    uint32_t item[2];
    uint32_t counts[2];       // pending positions of the cluster, by round parity
    int err;
    uint32_t list[kTailCap];
};

template <typename T>
__global__ void __launch_bounds__(kBatThreads) shuffle_cluster_kernel(BatchedArgs a) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ClusterCtl ctl;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t rank = cl.block_rank(), C = cl.num_blocks();
    T *A = reinterpret_cast<T *>(smem);
    uint32_t *res = reinterpret_cast<uint32_t *>(smem + (size_t)kClChunkCap * sizeof(T));
    uint16_t *jt = reinterpret_cast<uint16_t *>(res + kClChunkCap);
    uint32_t *bm = reinterpret_cast<uint32_t *>(jt + kClChunkCap);
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    if (tid == 0) {
        ctl.err = 0;
        ctl.counts[0] = ctl.counts[1] = 0;
    }
    const uint32_t n_items = a.offsets ? a.n_arrays : 1u;
    for (uint32_t it = 0;; it++) {
        const uint32_t par = it & 1u;
        if (rank == 0 && tid == 0) ctl.item[par] = atomicAdd(&a.queue[2], 1u);
        cl.sync();
        const uint32_t s = *cl.map_shared_rank(&ctl.item[par], 0);
        if (s >= n_items) break;  // the same value in every CTA of the cluster
        uint64_t o0 = 0, o1 = a.single_n, seed = a.single_seed;
        if (a.offsets) {
            o0 = a.offsets[s];
            o1 = a.offsets[s + 1];
            seed = a.seeds[s];
        }
        if (o1 < o0 || o1 - o0 > a.max_len) continue;  // reported by the per-CTA kernel
        const uint32_t n = (uint32_t)(o1 - o0);
        if (!a.use_cluster || n <= a.smem_cap || n > C * kClChunkCap) continue;
        const uint32_t chunk = ((n + C - 1) / C + 31) & ~31u;
        const uint32_t lo = rank * chunk;
        const uint32_t hi = min(n, lo + chunk);
        const uint32_t mine = hi > lo ? hi - lo : 0;
        const uint32_t nwords = chunk / 32;
        T *g = static_cast<T *>(a.data) + o0;
        for (uint32_t x = tid; x < chunk; x += blockDim.x) {
            if (x < mine) A[x] = g[lo + x];
            res[x] = 0;
        }
        for (uint32_t w = tid; w < nwords; w += blockDim.x) bm[w] = initial_pending_word(w, lo, n);
        if (tid == 0) {
            ctl.nseg = plan_segments(n, 1, a.nk, a.k_max, ctl.seg, kMaxSegs, &ctl.n_batches);
            if (ctl.nseg < 0) { ctl.nseg = 0; ctl.n_batches = 0; ctl.err = BRR_EINVAL; }
            ctl.counts[0] = ctl.counts[1] = 0;  // every read of the last array's counts is over
        }
        cl.sync();
        // batches are split evenly over the CTAs; each writes swap indices
        // into the CTA that owns the position
        const uint64_t g_lo = ctl.n_batches * rank / C, g_hi = ctl.n_batches * (rank + 1) / C;
        roll_plan_range(ctl.seg, ctl.nseg, g_lo, g_hi, seed, ctl.err, [&](uint32_t pos, uint32_t v) {
            const uint32_t o = pos / chunk;
            *(cl.map_shared_rank(jt, o) + (pos - o * chunk)) = (uint16_t)v;
        });
        cl.sync();
        if (a.j_out) {
            for (uint32_t x = tid; x < mine; x += blockDim.x) a.j_out[lo + x] = lo + x == 0 ? 0u : jt[x];
        }
        // owner CTA of global position j: j / chunk, by a multiply-high
        // (exact for j < 2^16 and chunk <= 2^13)
        const uint32_t magic = (uint32_t)((0xFFFFFFFFull + chunk) / chunk);
        auto slot = [&](uint32_t j) {
            const uint32_t o = __umulhi(j, magic);
            const uint32_t jl = j - o * chunk;
            return SlotRef<T>{cl.map_shared_rank(res, o) + jl, cl.map_shared_rank(A, o) + jl};
        };
        for (uint32_t round = 0;; round++) {
            if (round > n + 1) {  // cannot happen: every round commits a swap
                if (tid == 0) ctl.err = BRR_ETIMEOUT;
                break;
            }
            reserve_pass<T, uint16_t>(bm, nwords, jt, res, lo, slot);
            cl.sync();
            if (rank == 0 && tid == 0) ctl.counts[(round + 1) & 1u] = 0;
            const uint32_t pend = commit_pass<T, uint16_t>(bm, nwords, jt, A, res, lo, slot);
            if (lane == 0 && pend) atomicAdd(cl.map_shared_rank(&ctl.counts[round & 1u], 0), pend);
            cl.sync();
            const uint32_t left = *cl.map_shared_rank(&ctl.counts[round & 1u], 0);
            if (left == 0) break;
            if (left <= kTail) {
                // CTA 0's first warp finishes the few pending swaps in order
                if (rank == 0 && tid < 32) {
                    const uint32_t wpc = chunk / 32;  // bitmap words per CTA
                    finish_pending<T>(
                        C * wpc, ctl.list,
                        [&](uint32_t w) {
                            const uint32_t o = w / wpc;
                            return *(cl.map_shared_rank(bm, o) + (w - o * wpc));
                        },
                        [&](uint32_t p) {
                            const uint32_t o = __umulhi(p, magic);
                            return (uint32_t) * (cl.map_shared_rank(jt, o) + (p - o * chunk));
                        },
                        slot);
                }
                cl.sync();
                break;
            }
        }
        for (uint32_t x = tid; x < mine; x += blockDim.x) g[lo + x] = A[x];
    }
    // no CTA may leave while another can still read its shared memory
    cl.sync();
    if (tid == 0 && ctl.err) record_error(a.err, ctl.err);
}

// Per-CTA staging capacity for shared memory of `limit` bytes.
static uint32_t smem_capacity(size_t limit, uint32_t eb) {
    uint32_t cap = (uint32_t)std::min<size_t>(limit / (eb + 6), 65534);
    while (cap > 0 && smem_bytes_for(cap, eb) > limit) cap--;
    return cap;
}

template <typename T>
static size_t cluster_smem() {
    return (size_t)kClChunkCap * (sizeof(T) + 4 + 2) + kClChunkCap / 32 * 4;
}

template <typename T>
static cudaLaunchConfig_t cluster_config(cudaLaunchAttribute *attr, uint32_t clusters,
                                         cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClSize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(clusters * kClSize);
    cfg.blockDim = dim3(kBatThreads);
    cfg.dynamicSmemBytes = cluster_smem<T>();
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Kernel attributes and occupancy of the staged kernels, queried once per
// context and element size (these queries cost far more than a launch).
template <typename T>
static brr_status staged_setup(brr_ctx *ctx) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    if (ctx->staged_ready[ix]) return BRR_OK;
    const size_t smem_limit = (size_t)ctx->max_smem_optin - sizeof(BatchCtl) - 1024;
    const uint32_t cap = smem_capacity(smem_limit, sizeof(T));
    const size_t smem = smem_bytes_for(cap, sizeof(T));
    const void *kern = (const void *)shuffle_batched_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 0, per_sm_long = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatThreads, smem);
    if (e != cudaSuccess || per_sm < 1) return BRR_ECUDA;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_long, shuffle_long_kernel<T>, kLongThreads,
                                                      kLongBitmapSmem);
    if (e != cudaSuccess || per_sm_long < 1) return BRR_ECUDA;
    const void *ckern = (const void *)shuffle_cluster_kernel<T>;
    e = cudaFuncSetAttribute(ckern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_smem<T>());
    if (e != cudaSuccess) return cuda_status(e);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config<T>(attr, 1, 0);
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, ckern, &cfg);
    if (e != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        return BRR_ECUDA;
    }
    ctx->staged_cap[ix] = cap;
    ctx->staged_per_sm[ix] = per_sm;
    ctx->long_per_sm[ix] = per_sm_long;
    ctx->staged_clusters[ix] = clusters;
    ctx->staged_ready[ix] = true;
    return BRR_OK;
}

// Shared by brr_shuffle_batched (offsets != nullptr) and by brr_shuffle for
// arrays up to the cluster capacity (offsets == nullptr, one array).
template <typename T>
static brr_status launch_shuffle_staged(brr_ctx *ctx, BatchedArgs a, uint64_t max_len,
                                        cudaStream_t stream) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    brr_status st = staged_setup<T>(ctx);
    if (st != BRR_OK) return st;
    const uint32_t n_items = a.offsets ? a.n_arrays : 1u;
    a.max_len = (uint32_t)max_len;
    a.err = ctx->d_err;
    a.smem_cap = ctx->staged_cap[ix];
    a.cluster_cap = kClusterCap;
    // One array longer than a CTA's shared memory: a thread-block cluster
    // gives it the shared memory of 8 SMs (lowest latency; measured 0.26 ms
    // against 1.95 ms for one CTA working in L2 at n = 65,536).  Many arrays:
    // one CTA per array keeps every SM busy (measured 53 ms against 122 ms for
    // 65,536 arrays of log-uniform length in [16, 65,536]).
    a.use_cluster = n_items == 1 ? 1u : 0u;
    const size_t smem = smem_bytes_for(a.smem_cap, sizeof(T));
    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)ctx->staged_per_sm[ix] * ctx->num_sms, n_items);
    // one scratch slice per CTA of the long kernel: reservation words, swap
    // indices and pending bitmap of an array of up to max_len elements
    uint32_t long_grid = 0;
    if (max_len > a.smem_cap && !(a.use_cluster && max_len <= a.cluster_cap)) {
        a.slot_words = ((size_t)2 * max_len + (max_len + 31) / 32 + 63) & ~(size_t)63;
        const size_t budget = (size_t)2 << 30;
        long_grid = (uint32_t)std::max<size_t>(
            1, std::min<size_t>({(size_t)ctx->long_per_sm[ix] * ctx->num_sms, (size_t)n_items,
                                 budget / (a.slot_words * 4)}));
    }
    st = ensure_scratch(ctx, 256 + (size_t)long_grid * a.slot_words * 4, stream);
    if (st != BRR_OK) return st;
    char *base = static_cast<char *>(ctx->scratch);
    a.queue = reinterpret_cast<uint32_t *>(base);
    a.slot_res = reinterpret_cast<uint32_t *>(base + 256);
    cudaError_t e = cudaMemsetAsync(a.queue, 0, 4 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (a.use_cluster && max_len > a.smem_cap) {
        const uint32_t clusters = std::max<uint32_t>(
            1, std::min<uint32_t>((uint32_t)ctx->staged_clusters[ix], n_items));
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config<T>(attr, clusters, stream);
        e = cudaLaunchKernelEx(&cfg, shuffle_cluster_kernel<T>, a);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (long_grid) {
        const size_t bm_bytes = ((size_t)max_len + 31) / 32 * 4;
        a.long_bm_smem = bm_bytes <= kLongBitmapSmem ? 1u : 0u;
        shuffle_long_kernel<T><<<long_grid, kLongThreads, a.long_bm_smem ? bm_bytes : 0, stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    // the short kernel also validates every array
    shuffle_batched_kernel<T><<<grid, kBatThreads, smem, stream>>>(a);
    return cuda_status(cudaGetLastError());
}

brr_status launch_shuffle_batched(brr_ctx *ctx, void *data, const uint64_t *offsets,
                                  uint32_t n_arrays, uint32_t elem_bytes, const uint64_t *seeds,
                                  uint64_t max_len, const brr_schedule *sched,
                                  cudaStream_t stream) {
    BatchedArgs a = {};
    a.data = data;
    a.offsets = offsets;
    a.seeds = seeds;
    a.n_arrays = n_arrays;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = sched->n_k[k];
    a.k_max = sched->k_max;
    return elem_bytes == 4 ? launch_shuffle_staged<uint32_t>(ctx, a, max_len, stream)
                           : launch_shuffle_staged<uint64_t>(ctx, a, max_len, stream);
}

brr_status launch_shuffle_one_staged(brr_ctx *ctx, void *data, uint64_t n, uint32_t elem_bytes,
                                     uint64_t seed, const brr_schedule *sched, uint32_t *j_out,
                                     cudaStream_t stream) {
    BatchedArgs a = {};
    a.data = data;
    a.n_arrays = 1;
    a.single_n = (uint32_t)n;
    a.single_seed = seed;
    a.j_out = j_out;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = sched->n_k[k];
    a.k_max = sched->k_max;
    return elem_bytes == 4 ? launch_shuffle_staged<uint32_t>(ctx, a, n, stream)
                           : launch_shuffle_staged<uint64_t>(ctx, a, n, stream);
}

uint64_t staged_shuffle_cap() { return kClusterCap; }

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
    brr_status st = ensure_scratch(ctx, 256 + (size_t)a.n_slots * a.slot_words * 4, stream);
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
