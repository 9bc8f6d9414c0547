// chains.cu -- applying the swaps of a Fisher-Yates shuffle (Algorithm 1)
// by chain resolution: no rounds, four parallel passes.
//
// The sequential loop "for p = n-1 .. 1: exchange A[p], A[j[p]]" has a closed
// form.  Slot y is written by the steps c > y that target it (in sequential,
// i.e. decreasing, order) and then by step y itself, after which slot y is
// final.  Step c moves whatever slot j_c holds into its final place c.  That
// is the value the previous step targeting j_c -- the next larger member
// succ(c) of the group of steps with target j_c -- carried in: the value slot
// succ(c) held just before step succ(c), W(succ(c)).  Without such a step
// slot j_c still holds its initial value j_c.  In the same way W(x) = W(parent(x))
// where parent(x) is the smallest step above x that targets x, and W(x) = x
// when there is none.  With step 0 a no-op:
//
//     final[c] = A[W(succ(c))], or A[j_c] if c is the largest step with target j_c
//     final[0] = A[W(0)]
//     W(x)     = the root of x in the forest x -> parent(x), parent(x) > x.
//
// Passes (each fully parallel, separated by a barrier):
//  1. roll every batch of the plan (Algorithm 4) and push step c onto the
//     list of target j_c: one atomic exchange of the list head, the old head
//     becomes c's link (no ordering is needed until the barrier);
//  2. per target y: sort the list ascending in place (steps were pushed in
//     roughly decreasing order, so it is nearly sorted already); parent(y)
//     is its first member above y (the head, or the next one when the head
//     is y itself); the last member's link is set to y, so afterwards a link
//     > its position is a successor and a link <= its position is that
//     step's target;
//  3. per x, in decreasing order: replace parent(x) by the root (path
//     compression; parents are larger, so they are mostly finished already);
//  4. per position c: gather final[c] from the original array.
//
// Three tiers share the passes through an index-space accessor: one CTA with
// 16-bit links in its shared memory; one thread-block cluster with the links
// and elements spread over the CTAs' shared memory (16-bit links, n <= 65,536);
// global memory with 32-bit links in scratch (one CTA, or the whole grid in
// separate launches).  Every loop is bounded by the array length; a bound
// that runs out records BRR_ETIMEOUT instead of looping.
#include <algorithm>

#include <cooperative_groups.h>

#include "brr_common.cuh"
#include "internal.h"

namespace brr {

constexpr int kChainThreads = 512;             // CTA, cluster and long kernels
constexpr int kChainGridThreads = 256;         // global-memory grid kernels
constexpr uint32_t kChainClusterCap = 65536;   // 16-bit links
constexpr int kChainClusterBatched = 4;        // CTAs per cluster, batched calls
constexpr int kChainClusterSingle = 8;         // CTAs per cluster, one array

// ------------------------------------------------------ index spaces --
__device__ __forceinline__ uint32_t cta_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-bit links in this CTA's shared memory (shared::cta addresses).
struct CtaIdx {
    uint32_t head, next;
    __device__ __forceinline__ uint32_t hp(uint32_t y) const { return head + 2u * y; }
    __device__ __forceinline__ uint32_t np(uint32_t c) const { return next + 2u * c; }
    // exchange of a 16-bit head; a failed CAS means another push succeeded
    static __device__ __forceinline__ uint32_t exch(uint32_t a, uint32_t v, uint32_t limit, bool &ok) {
        uint32_t cur = ld(a);
        for (uint32_t it = 0; it < limit; it++) {
            uint16_t prev;
            asm volatile("atom.relaxed.cta.shared::cta.cas.b16 %0, [%1], %2, %3;"
                         : "=h"(prev) : "r"(a), "h"((uint16_t)cur), "h"((uint16_t)v) : "memory");
            if (prev == cur) return cur;
            cur = prev;
        }
        ok = false;
        return cur;
    }
    static __device__ __forceinline__ uint32_t ld(uint32_t a) {
        uint16_t v;
        asm volatile("ld.shared::cta.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
        return v;
    }
    static __device__ __forceinline__ void st(uint32_t a, uint32_t v) {
        asm volatile("st.shared::cta.u16 [%0], %1;" ::"r"(a), "h"((uint16_t)v) : "memory");
    }
};

__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// 16-bit links spread over the CTAs of a cluster: positions [r*chunk,
// (r+1)*chunk) live in CTA r at the same shared-memory offsets
// (shared::cluster addresses).  owner(x) = x / chunk by a multiply-high,
// exact for x < 2^16 and chunk <= 2^16.
struct ClusterIdx {
    uint32_t head, next;  // this CTA's shared::cta addresses of the arrays
    uint32_t chunk, magic;
    __device__ __forceinline__ uint32_t owner(uint32_t x) const { return __umulhi(x, magic); }
    __device__ __forceinline__ uint32_t at(uint32_t base, uint32_t x) const {
        const uint32_t o = owner(x);
        return mapa(base + 2u * (x - o * chunk), o);
    }
    __device__ __forceinline__ uint32_t hp(uint32_t y) const { return at(head, y); }
    __device__ __forceinline__ uint32_t np(uint32_t c) const { return at(next, c); }
    static __device__ __forceinline__ uint32_t exch(uint32_t a, uint32_t v, uint32_t limit, bool &ok) {
        uint32_t cur = ld(a);
        for (uint32_t it = 0; it < limit; it++) {
            uint16_t prev;
            asm volatile("atom.relaxed.cluster.shared::cluster.cas.b16 %0, [%1], %2, %3;"
                         : "=h"(prev) : "r"(a), "h"((uint16_t)cur), "h"((uint16_t)v) : "memory");
            if (prev == cur) return cur;
            cur = prev;
        }
        ok = false;
        return cur;
    }
    static __device__ __forceinline__ uint32_t ld(uint32_t a) {
        uint16_t v;
        asm volatile("ld.shared::cluster.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
        return v;
    }
    static __device__ __forceinline__ void st(uint32_t a, uint32_t v) {
        asm volatile("st.shared::cluster.u16 [%0], %1;" ::"r"(a), "h"((uint16_t)v) : "memory");
    }
};

// 32-bit links in global memory; the head exchanges are atomic at CTA scope
// (one CTA owns the lists) or GPU scope (the whole grid pushes).
template <bool kGpu>
struct GlobalIdx {
    uint32_t *head, *next;
    __device__ __forceinline__ uint32_t *hp(uint32_t y) const { return head + y; }
    __device__ __forceinline__ uint32_t *np(uint32_t c) const { return next + c; }
    static __device__ __forceinline__ uint32_t exch(uint32_t *a, uint32_t v, uint32_t, bool &) {
        uint32_t old;
        if (kGpu)
            asm volatile("atom.relaxed.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
        else
            asm volatile("atom.relaxed.cta.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
        return old;
    }
    static __device__ __forceinline__ uint32_t ld(const uint32_t *a) {
        uint32_t v;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
        return v;
    }
    static __device__ __forceinline__ void st(uint32_t *a, uint32_t v) {
        asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
    }
};

// ----------------------------------------------------------- the passes --
// Pass 1: push step c (1 <= c < n) onto the list of target y.
template <class Ix>
__device__ __forceinline__ bool chain_push(const Ix &ix, uint32_t c, uint32_t y, uint32_t limit) {
    bool ok = true;
    const uint32_t old = Ix::exch(ix.hp(y), c, limit, ok);
    Ix::st(ix.np(c), old);
    return ok;
}

// Pass 2: sort y's list ascending in place (insertion: appended at the tail
// when larger than it, as almost always, else linked in by a walk of the
// sorted part); then head[y] <- parent of y (y itself when it has none) and
// the last member's link <- y.  Only the walker of y touches y's members.
template <class Ix>
__device__ __forceinline__ bool chain_sort(const Ix &ix, uint32_t y, uint32_t limit) {
    const auto hp = ix.hp(y);
    uint32_t first = 0, last = 0;
    uint32_t it = 0;
    for (uint32_t m = Ix::ld(hp); m != 0u;) {
        if (++it > limit) return false;
        const auto mp = ix.np(m);
        const uint32_t nx = Ix::ld(mp);  // next unsorted member
        if (first == 0u) {
            first = last = m;
        } else if (m > last) {
            Ix::st(ix.np(last), m);
            last = m;
        } else if (m < first) {
            Ix::st(mp, first);
            first = m;
        } else {
            // first < m < last: the sorted links from first reach a member
            // above m no later than last
            uint32_t p = first;
            for (;;) {
                if (++it > limit) return false;
                const uint32_t q = Ix::ld(ix.np(p));
                if (q > m) {
                    Ix::st(mp, q);
                    Ix::st(ix.np(p), m);
                    break;
                }
                p = q;
            }
        }
        m = nx;
    }
    uint32_t par = first;
    if (first != 0u) {
        if (first == y) par = first == last ? 0u : Ix::ld(ix.np(first));  // y targets itself
        Ix::st(ix.np(last), y);
    }
    Ix::st(hp, par != 0u ? par : y);
    return true;
}

// Pass 3: head[x] <- root of x.  Any value read is x's parent or a larger
// ancestor (compression only moves entries toward their roots), and a root
// is the only entry equal to its index, so the walk strictly increases.
template <class Ix>
__device__ __forceinline__ bool chain_root(const Ix &ix, uint32_t x, uint32_t limit) {
    const auto qp = ix.hp(x);
    uint32_t r = Ix::ld(qp);
    if (r == x) return true;
    for (uint32_t it = 0;; it++) {
        if (it >= limit) return false;
        const uint32_t q = Ix::ld(ix.hp(r));
        if (q == r) break;
        r = q;
    }
    Ix::st(qp, r);
    return true;
}

// Pass 4: original index of the element that ends at position c.
template <class Ix>
__device__ __forceinline__ uint32_t chain_source(const Ix &ix, uint32_t c) {
    if (c == 0u) return Ix::ld(ix.hp(0));
    const uint32_t l = Ix::ld(ix.np(c));
    return l > c ? Ix::ld(ix.hp(l)) : l;
}

__host__ __device__ __forceinline__ uint32_t chain_limit(uint64_t n) {
    return n >= 0x7FFFFFFEull ? 0xFFFFFFFFu : (uint32_t)(2 * n + 2);
}

// ---------------------------------------------------- per-array kernels --
struct ChainCtl {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
    int err;
    uint32_t item[2];
};

struct ChainArgs {
    void *data;
    const uint64_t *offsets;  // nullptr: one array of single_n elements
    const uint64_t *seeds;
    uint32_t n_arrays;
    uint64_t nk[BRR_SCHED_KMAX + 1];
    uint32_t k_max;
    uint32_t cta_full_cap; // arrays up to this: one CTA, elements and links in shared memory
    uint32_t cta_cap;      // up to this: one CTA, links in shared memory, elements
                           //   gathered from a copy in the CTA's global slot
    uint32_t cluster_cap;  // up to cluster_cap: one cluster; longer: chain_long_kernel
    uint32_t chunk_cap;    // positions per CTA of the cluster kernel
    uint32_t max_len;
    uint32_t *queue;       // [3]: next array of the CTA, cluster and long kernels
    unsigned char *cta_slots;   // CTA kernel: per CTA, a copy of the array
    size_t cta_slot_bytes;
    unsigned char *slots;       // long kernel: per CTA, links and a copy of the array
    size_t slot_bytes;
    uint32_t single_n;
    uint64_t single_seed;
    uint32_t *j_out;       // single-array form: swap indices (optional)
    int *err;
};

// Bounds and seed of array s; false if the offsets are invalid or the array
// is longer than max_len.
__device__ __forceinline__ bool chain_item(const ChainArgs &a, uint32_t s, uint64_t &o0,
                                           uint64_t &len, uint64_t &seed) {
    if (!a.offsets) {
        o0 = 0;
        len = a.single_n;
        seed = a.single_seed;
        return true;
    }
    o0 = a.offsets[s];
    const uint64_t o1 = a.offsets[s + 1];
    seed = a.seeds[s];
    if (o1 < o0) return false;
    len = o1 - o0;
    return len <= a.max_len;
}

__device__ __forceinline__ void chain_plan(ChainCtl &ctl, const ChainArgs &a, uint32_t n) {
    ctl.nseg = plan_segments(n, 1, a.nk, a.k_max, ctl.seg, kMaxSegs, &ctl.n_batches);
    if (ctl.nseg < 0) {
        ctl.err = BRR_EINVAL;
        ctl.nseg = 0;
        ctl.n_batches = 0;
    }
}

// Shared memory of the CTA kernel for an array of n elements of eb bytes
// (eb = 0: links only).
__host__ __device__ __forceinline__ size_t chain_cta_smem(uint32_t n, uint32_t eb) {
    return (((size_t)n * eb + 15) & ~(size_t)15) + 2 * (((size_t)n + 7) & ~(size_t)7) * 2;
}

// Arrays of 2 .. cta_cap elements: one CTA per array at a time with the links
// in shared memory, and the elements too up to cta_full_cap; longer arrays
// are copied to the CTA's global slot (resident in L2) and gathered from
// there.  Also validates every array (lengths above max_len or decreasing
// offsets record BRR_EINVAL).
template <typename T>
__global__ void __launch_bounds__(kChainThreads) chain_cta_kernel(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ChainCtl ctl;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) ctl.err = 0;
    const uint32_t n_items = a.offsets ? a.n_arrays : 1u;
    for (;;) {
        __syncthreads();
        if (tid == 0) ctl.item[0] = atomicAdd(&a.queue[0], 1u);
        __syncthreads();
        const uint32_t s = ctl.item[0];
        if (s >= n_items) break;
        uint64_t o0, len, seed;
        if (!chain_item(a, s, o0, len, seed)) {
            if (tid == 0) ctl.err = BRR_EINVAL;
            continue;
        }
        if (len < 2 || len > a.cta_cap) continue;
        const uint32_t n = (uint32_t)len;
        if (tid == 0) chain_plan(ctl, a, n);
        T *g = static_cast<T *>(a.data) + o0;
        const bool staged = n <= a.cta_full_cap;
        T *As = staged ? reinterpret_cast<T *>(smem)
                       : reinterpret_cast<T *>(a.cta_slots + (size_t)blockIdx.x * a.cta_slot_bytes);
        uint16_t *head = reinterpret_cast<uint16_t *>(
            smem + (staged ? (((size_t)n * sizeof(T) + 15) & ~(size_t)15) : 0));
        uint16_t *next = head + ((n + 7) & ~7u);
        for (uint32_t x = tid; x < n; x += blockDim.x) {
            As[x] = g[x];
            head[x] = 0;
            next[x] = 0;
        }
        __syncthreads();
        if (ctl.nseg == 0) continue;
        const CtaIdx ix{cta_addr(head), cta_addr(next)};
        const uint32_t lim = chain_limit(n);
        uint32_t *jo = a.j_out;
        bool ok = true;
        roll_plan_range(ctl.seg, ctl.nseg, 0, ctl.n_batches, seed, ctl.err, [&](uint32_t pos, uint32_t v) {
            if (jo) jo[pos] = v;
            ok = chain_push(ix, pos, v, lim) && ok;
        });
        if (jo && tid == 0) jo[0] = 0;
        __syncthreads();
        for (uint32_t y = tid; y < n; y += blockDim.x) ok = chain_sort(ix, y, lim) && ok;
        __syncthreads();
        for (int32_t x = (int32_t)n - 1 - (int32_t)tid; x >= 0; x -= (int32_t)blockDim.x)
            ok = chain_root(ix, (uint32_t)x, lim) && ok;
        __syncthreads();
        for (uint32_t c = tid; c < n; c += blockDim.x) g[c] = As[chain_source(ix, c)];
        if (!ok) ctl.err = BRR_ETIMEOUT;
    }
    __syncthreads();
    if (tid == 0 && ctl.err) record_error(a.err, ctl.err);
}

template <typename T> __device__ __forceinline__ T ld_cluster(uint32_t a);
template <> __device__ __forceinline__ uint32_t ld_cluster<uint32_t>(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
template <> __device__ __forceinline__ uint64_t ld_cluster<uint64_t>(uint32_t a) {
    uint64_t v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}

// Arrays of cta_cap+1 .. C*chunk_cap elements (single-array form: any length
// up to that): one thread-block cluster per array.  CTA r holds positions
// [r*chunk, (r+1)*chunk): elements, heads and links, at the same offsets in
// every CTA; the batches are split evenly over the CTAs.
template <typename T>
__global__ void __launch_bounds__(kChainThreads) chain_cluster_kernel(ChainArgs a) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ChainCtl ctl;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t rank = cl.block_rank(), C = cl.num_blocks();
    const uint32_t tid = threadIdx.x;
    T *As = reinterpret_cast<T *>(smem);
    uint16_t *head = reinterpret_cast<uint16_t *>(smem + (size_t)a.chunk_cap * sizeof(T));
    uint16_t *next = head + a.chunk_cap;
    const uint32_t as_addr = cta_addr(As);
    if (tid == 0) ctl.err = 0;
    const uint32_t n_items = a.offsets ? a.n_arrays : 1u;
    for (uint32_t it = 0;; it++) {
        const uint32_t par = it & 1u;
        if (rank == 0 && tid == 0) ctl.item[par] = atomicAdd(&a.queue[1], 1u);
        cl.sync();
        const uint32_t s = *cl.map_shared_rank(&ctl.item[par], 0);
        if (s >= n_items) break;  // the same value in every CTA of the cluster
        uint64_t o0, len, seed;
        if (!chain_item(a, s, o0, len, seed)) continue;  // reported by the CTA kernel
        if (len < 2 || (a.offsets && len <= a.cta_cap) || len > (uint64_t)C * a.chunk_cap) continue;
        const uint32_t n = (uint32_t)len;
        const uint32_t chunk = ((n + C - 1) / C + 7) & ~7u;
        const uint32_t lo = rank * chunk;
        const uint32_t hi = min(n, lo + chunk);
        T *g = static_cast<T *>(a.data) + o0;
        for (uint32_t x = tid; x < chunk; x += blockDim.x) {
            if (lo + x < hi) As[x] = g[lo + x];
            head[x] = 0;
            next[x] = 0;
        }
        if (tid == 0) chain_plan(ctl, a, n);
        cl.sync();
        if (ctl.nseg == 0) continue;  // the same plan in every CTA
        const ClusterIdx ix{cta_addr(head), cta_addr(next), chunk,
                            (uint32_t)((0xFFFFFFFFull + chunk) / chunk)};
        const uint32_t lim = chain_limit(n);
        uint32_t *jo = a.j_out;
        bool ok = true;
        const uint64_t g_lo = ctl.n_batches * rank / C, g_hi = ctl.n_batches * (rank + 1) / C;
        roll_plan_range(ctl.seg, ctl.nseg, g_lo, g_hi, seed, ctl.err, [&](uint32_t pos, uint32_t v) {
            if (jo) jo[pos] = v;
            ok = chain_push(ix, pos, v, lim) && ok;
        });
        if (jo && rank == 0 && tid == 0) jo[0] = 0;
        cl.sync();
        for (uint32_t y = lo + tid; y < hi; y += blockDim.x) ok = chain_sort(ix, y, lim) && ok;
        cl.sync();
        for (int32_t x = (int32_t)hi - 1 - (int32_t)tid; x >= (int32_t)lo; x -= (int32_t)blockDim.x)
            ok = chain_root(ix, (uint32_t)x, lim) && ok;
        cl.sync();
        for (uint32_t c = lo + tid; c < hi; c += blockDim.x) {
            const uint32_t src = chain_source(ix, c);
            const uint32_t o = ix.owner(src);
            g[c] = ld_cluster<T>(mapa(as_addr + (uint32_t)sizeof(T) * (src - o * chunk), o));
        }
        if (!ok) ctl.err = BRR_ETIMEOUT;
    }
    // no CTA may leave while another can still read its shared memory
    cl.sync();
    if (tid == 0 && ctl.err) record_error(a.err, ctl.err);
}

// Layout of one long-kernel slot: heads, links (32-bit) and a copy of the
// array, for arrays of up to max_len elements.
__host__ __device__ __forceinline__ size_t chain_slot_bytes(uint64_t max_len, uint32_t eb) {
    const size_t links = ((size_t)max_len * 4 + 255) & ~(size_t)255;
    return 2 * links + (((size_t)max_len * eb + 255) & ~(size_t)255);
}

// Batched arrays longer than cluster_cap: one CTA per array in global
// memory, with scratch slot blockIdx.x (resident in L2 while it is used).
template <typename T>
__global__ void __launch_bounds__(kChainThreads) chain_long_kernel(ChainArgs a) {
    __shared__ ChainCtl ctl;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) ctl.err = 0;
    const uint32_t n_items = a.offsets ? a.n_arrays : 1u;
    const size_t links = ((size_t)a.max_len * 4 + 255) & ~(size_t)255;
    unsigned char *slot = a.slots + (size_t)blockIdx.x * a.slot_bytes;
    uint32_t *head = reinterpret_cast<uint32_t *>(slot);
    uint32_t *next = reinterpret_cast<uint32_t *>(slot + links);
    T *copy = reinterpret_cast<T *>(slot + 2 * links);
    for (;;) {
        __syncthreads();
        if (tid == 0) ctl.item[0] = atomicAdd(&a.queue[2], 1u);
        __syncthreads();
        const uint32_t s = ctl.item[0];
        if (s >= n_items) break;
        uint64_t o0, len, seed;
        if (!chain_item(a, s, o0, len, seed)) continue;  // reported by the CTA kernel
        if (len <= a.cluster_cap) continue;
        const uint32_t n = (uint32_t)len;
        if (tid == 0) chain_plan(ctl, a, n);
        T *g = static_cast<T *>(a.data) + o0;
        for (uint32_t x = tid; x < n; x += blockDim.x) {
            copy[x] = g[x];
            head[x] = 0;
            next[x] = 0;
        }
        __syncthreads();
        if (ctl.nseg == 0) continue;
        const GlobalIdx<false> ix{head, next};
        const uint32_t lim = chain_limit(n);
        bool ok = true;
        roll_plan_range(ctl.seg, ctl.nseg, 0, ctl.n_batches, seed, ctl.err,
                        [&](uint32_t pos, uint32_t v) { ok = chain_push(ix, pos, v, lim) && ok; });
        __syncthreads();
        for (uint32_t y = tid; y < n; y += blockDim.x) ok = chain_sort(ix, y, lim) && ok;
        __syncthreads();
        for (int64_t x = (int64_t)n - 1 - tid; x >= 0; x -= blockDim.x) ok = chain_root(ix, (uint32_t)x, lim) && ok;
        __syncthreads();
        for (uint32_t c = tid; c < n; c += blockDim.x) g[c] = copy[chain_source(ix, c)];
        if (!ok) ctl.err = BRR_ETIMEOUT;
    }
    __syncthreads();
    if (tid == 0 && ctl.err) record_error(a.err, ctl.err);
}

// ------------------------------------------------- one array, whole grid --
struct ChainGridArgs {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
    uint64_t seed;
    uint32_t *head, *next;
    uint32_t n;
    uint32_t *j_out;
    int *err;
};

__global__ void __launch_bounds__(kChainGridThreads) chain_grid_push(ChainGridArgs a) {
    const GlobalIdx<true> ix{a.head, a.next};
    const uint32_t lim = chain_limit(a.n);
    bool ok = true, rolled = true;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n_batches; g += stride)
        rolled = roll_plan_batch(a.seg, a.nseg, g, a.seed, [&](uint32_t pos, uint32_t v) {
                     if (a.j_out) a.j_out[pos] = v;
                     ok = chain_push(ix, pos, v, lim) && ok;
                 }) && rolled;
    if (a.j_out && blockIdx.x == 0 && threadIdx.x == 0) a.j_out[0] = 0;
    if (!rolled) record_error(a.err, BRR_ERETRY);
    if (!ok) record_error(a.err, BRR_ETIMEOUT);
}

__global__ void __launch_bounds__(kChainGridThreads) chain_grid_sort(ChainGridArgs a) {
    const GlobalIdx<true> ix{a.head, a.next};
    const uint32_t lim = chain_limit(a.n);
    bool ok = true;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < a.n; y += stride)
        ok = chain_sort(ix, y, lim) && ok;
    if (!ok) record_error(a.err, BRR_ETIMEOUT);
}

__global__ void __launch_bounds__(kChainGridThreads) chain_grid_root(ChainGridArgs a) {
    const GlobalIdx<true> ix{a.head, a.next};
    const uint32_t lim = chain_limit(a.n);
    bool ok = true;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)a.n - 1 - ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); x >= 0; x -= stride)
        ok = chain_root(ix, (uint32_t)x, lim) && ok;
    if (!ok) record_error(a.err, BRR_ETIMEOUT);
}

template <typename T>
__global__ void __launch_bounds__(kChainGridThreads)
chain_grid_gather(ChainGridArgs a, const T *__restrict__ copy, T *__restrict__ A) {
    const GlobalIdx<true> ix{a.head, a.next};
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < a.n; c += stride)
        A[c] = copy[chain_source(ix, c)];
}

// ------------------------------------------------------------ launchers --
template <typename T>
static cudaLaunchConfig_t chain_cluster_config(cudaLaunchAttribute *attr, uint32_t csize,
                                               uint32_t clusters, uint32_t chunk_cap,
                                               cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(clusters * csize);
    cfg.blockDim = dim3(kChainThreads);
    cfg.dynamicSmemBytes = (size_t)chunk_cap * (sizeof(T) + 4);
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Kernel attributes and occupancy, once per context and element size.
template <typename T>
static brr_status chain_setup(brr_ctx *ctx) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    if (ctx->chain_ready[ix]) return BRR_OK;
    const size_t limit = (size_t)ctx->max_smem_optin - sizeof(ChainCtl) - 1024;
    uint32_t full = (uint32_t)std::min<size_t>(limit / (sizeof(T) + 4), kChainClusterCap);
    while (full > 0 && chain_cta_smem(full, sizeof(T)) > limit) full--;
    uint32_t cap = (uint32_t)std::min<size_t>(limit / 4, kChainClusterCap);
    while (cap > 0 && chain_cta_smem(cap, 0) > limit) cap--;
    const size_t smem = std::max(chain_cta_smem(full, sizeof(T)), chain_cta_smem(cap, 0));
    const void *kc = (const void *)chain_cta_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 0, long_per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kc, kChainThreads, smem);
    if (e != cudaSuccess || per_sm < 1) return BRR_ECUDA;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&long_per_sm, chain_long_kernel<T>, kChainThreads, 0);
    if (e != cudaSuccess || long_per_sm < 1) return BRR_ECUDA;
    const void *kcl = (const void *)chain_cluster_kernel<T>;
    const uint32_t caps[2] = {kChainClusterCap / kChainClusterBatched, kChainClusterCap / kChainClusterSingle};
    e = cudaFuncSetAttribute(kcl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)caps[0] * (sizeof(T) + 4)));
    if (e != cudaSuccess) return cuda_status(e);
    int clusters[2] = {0, 0};
    const uint32_t sizes[2] = {kChainClusterBatched, kChainClusterSingle};
    for (int i = 0; i < 2; i++) {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = chain_cluster_config<T>(attr, sizes[i], 1, caps[i], 0);
        e = cudaOccupancyMaxActiveClusters(&clusters[i], kcl, &cfg);
        if (e != cudaSuccess || clusters[i] < 1) {
            cudaGetLastError();
            return BRR_ECUDA;
        }
    }
    ctx->chain_cta_full_cap[ix] = full;
    ctx->chain_cta_cap[ix] = cap;
    ctx->chain_cta_smem[ix] = smem;
    ctx->chain_cta_per_sm[ix] = per_sm;
    ctx->chain_long_per_sm[ix] = long_per_sm;
    ctx->chain_clusters[ix][0] = clusters[0];
    ctx->chain_clusters[ix][1] = clusters[1];
    ctx->chain_ready[ix] = true;
    return BRR_OK;
}

// Batched shuffles (offsets != nullptr), or one array (offsets == nullptr)
// of at most kChainClusterCap elements.  Which kernel takes an array:
//   batched: n <= cta_cap                 chain_cta_kernel
//            n <= 65,536, tune.batched_cluster = 1: chain_cluster_kernel, 4 CTAs
//            longer                       chain_long_kernel
//   one:     n <= tune.single_cta_max     chain_cta_kernel (one CTA)
//            otherwise                    chain_cluster_kernel, 8 CTAs
template <typename T>
static brr_status launch_chains_staged(brr_ctx *ctx, ChainArgs a, uint64_t max_len, bool single_cta,
                                       cudaStream_t stream) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    brr_status st = chain_setup<T>(ctx);
    if (st != BRR_OK) return st;
    const bool single = a.offsets == nullptr;
    const uint32_t n_items = single ? 1u : a.n_arrays;
    a.max_len = (uint32_t)max_len;
    a.err = ctx->d_err;
    a.cta_full_cap = ctx->chain_cta_full_cap[ix];
    a.cta_cap = ctx->chain_cta_cap[ix];
    const bool use_cta = single ? single_cta : true;
    const bool use_cluster = single ? !single_cta
                                    : (ctx->tune.batched_cluster != 0 && max_len > a.cta_cap);
    a.cluster_cap = single ? kChainClusterCap : (ctx->tune.batched_cluster ? kChainClusterCap : a.cta_cap);
    const uint32_t csize = single ? kChainClusterSingle : kChainClusterBatched;
    a.chunk_cap = kChainClusterCap / csize;
    const uint32_t cta_grid = (uint32_t)std::min<uint64_t>((uint64_t)ctx->chain_cta_per_sm[ix] * ctx->num_sms, n_items);
    // global slots: copies of the arrays the CTA kernel cannot stage, and
    // links + copies of the arrays the long kernel takes
    size_t cta_slots = 0;
    if (use_cta && max_len > a.cta_full_cap) {
        a.cta_slot_bytes = ((size_t)std::min<uint64_t>(max_len, a.cta_cap) * sizeof(T) + 255) & ~(size_t)255;
        cta_slots = (size_t)cta_grid * a.cta_slot_bytes;
    }
    uint32_t long_grid = 0;
    if (!single && max_len > a.cluster_cap) {
        a.slot_bytes = chain_slot_bytes(max_len, sizeof(T));
        const size_t budget = (size_t)2 << 30;
        long_grid = (uint32_t)std::max<size_t>(
            1, std::min<size_t>({(size_t)ctx->chain_long_per_sm[ix] * ctx->num_sms, (size_t)n_items,
                                 budget / a.slot_bytes}));
    }
    st = ensure_scratch(ctx, 256 + cta_slots + (size_t)long_grid * a.slot_bytes);
    if (st != BRR_OK) return st;
    unsigned char *base = static_cast<unsigned char *>(ctx->scratch);
    a.queue = reinterpret_cast<uint32_t *>(base);
    a.cta_slots = base + 256;
    a.slots = base + 256 + cta_slots;
    cudaError_t e = cudaMemsetAsync(a.queue, 0, 4 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (use_cluster) {
        const int ci = single ? 1 : 0;
        const uint32_t clusters = std::max<uint32_t>(
            1, std::min<uint32_t>((uint32_t)ctx->chain_clusters[ix][ci], n_items));
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = chain_cluster_config<T>(attr, csize, clusters, a.chunk_cap, stream);
        e = cudaLaunchKernelEx(&cfg, chain_cluster_kernel<T>, a);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (long_grid) {
        chain_long_kernel<T><<<long_grid, kChainThreads, 0, stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    if (use_cta) {
        chain_cta_kernel<T><<<cta_grid, kChainThreads, ctx->chain_cta_smem[ix], stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    return BRR_OK;
}

brr_status launch_chains_batched(brr_ctx *ctx, void *data, const uint64_t *offsets, uint32_t n_arrays,
                                 uint32_t elem_bytes, const uint64_t *seeds, uint64_t max_len,
                                 const brr_schedule *sched, cudaStream_t stream) {
    ChainArgs a = {};
    a.data = data;
    a.offsets = offsets;
    a.seeds = seeds;
    a.n_arrays = n_arrays;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = sched->n_k[k];
    a.k_max = sched->k_max;
    return elem_bytes == 4 ? launch_chains_staged<uint32_t>(ctx, a, max_len, false, stream)
                           : launch_chains_staged<uint64_t>(ctx, a, max_len, false, stream);
}

size_t chains_grid_scratch(uint64_t n, uint32_t elem_bytes) {
    const size_t links = ((size_t)n * 4 + 255) & ~(size_t)255;
    return 256 + 2 * links + (((size_t)n * elem_bytes + 255) & ~(size_t)255);
}

// One array of 65,537 .. 2^32 - 2 elements on `scratch` (chains_grid_scratch
// bytes): heads, links and a copy of the array.
brr_status launch_chains_grid(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                              const brr_schedule *sched, uint32_t *j_out, void *scratch, int *err,
                              int num_sms, cudaStream_t stream) {
    ChainGridArgs a;
    a.nseg = plan_segments(n, 1, sched->n_k, sched->k_max, a.seg, kMaxSegs, &a.n_batches);
    if (a.nseg < 0) return BRR_EINVAL;
    a.seed = seed;
    a.n = (uint32_t)n;
    a.j_out = j_out;
    a.err = err;
    const size_t links = ((size_t)n * 4 + 255) & ~(size_t)255;
    unsigned char *base = static_cast<unsigned char *>(scratch) + 256;
    a.head = reinterpret_cast<uint32_t *>(base);
    a.next = reinterpret_cast<uint32_t *>(base + links);
    void *copy = base + 2 * links;
    cudaError_t e = cudaMemsetAsync(base, 0, 2 * links, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(copy, data, (size_t)n * elem_bytes, cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return cuda_status(e);
    const uint64_t cap = (uint64_t)num_sms * 8;
    const unsigned g_ins = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(cap, (a.n_batches + kChainGridThreads - 1) / kChainGridThreads));
    const unsigned g_pos = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(cap, (n + kChainGridThreads - 1) / kChainGridThreads));
    chain_grid_push<<<g_ins, kChainGridThreads, 0, stream>>>(a);
    chain_grid_sort<<<g_pos, kChainGridThreads, 0, stream>>>(a);
    chain_grid_root<<<g_pos, kChainGridThreads, 0, stream>>>(a);
    if (elem_bytes == 4)
        chain_grid_gather<uint32_t><<<g_pos, kChainGridThreads, 0, stream>>>(
            a, static_cast<const uint32_t *>(copy), static_cast<uint32_t *>(data));
    else
        chain_grid_gather<uint64_t><<<g_pos, kChainGridThreads, 0, stream>>>(
            a, static_cast<const uint64_t *>(copy), static_cast<uint64_t *>(data));
    return cuda_status(cudaGetLastError());
}

// One array: one CTA up to tune.single_cta_max elements, one cluster of 8
// up to tune.single_cluster_max (at most 65,536), else the grid passes.
brr_status launch_chains_one(brr_ctx *ctx, void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                             const brr_schedule *sched, uint32_t *j_out, cudaStream_t stream) {
    const int ix = elem_bytes == 4 ? 0 : 1;
    brr_status st = elem_bytes == 4 ? chain_setup<uint32_t>(ctx) : chain_setup<uint64_t>(ctx);
    if (st != BRR_OK) return st;
    const bool cta = n <= std::min<uint64_t>(ctx->tune.single_cta_max, ctx->chain_cta_cap[ix]);
    const bool cluster = !cta && n <= std::min<uint64_t>(ctx->tune.single_cluster_max, kChainClusterCap);
    if (cta || cluster) {
        ChainArgs a = {};
        a.data = data;
        a.n_arrays = 1;
        a.single_n = (uint32_t)n;
        a.single_seed = seed;
        a.j_out = j_out;
        for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = sched->n_k[k];
        a.k_max = sched->k_max;
        return elem_bytes == 4 ? launch_chains_staged<uint32_t>(ctx, a, n, cta, stream)
                               : launch_chains_staged<uint64_t>(ctx, a, n, cta, stream);
    }
    st = ensure_scratch(ctx, chains_grid_scratch(n, elem_bytes));
    if (st != BRR_OK) return st;
    return launch_chains_grid(data, n, elem_bytes, seed, sched, j_out, ctx->scratch, ctx->d_err,
                              ctx->num_sms, stream);
}

}  // namespace brr
