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

constexpr int kChainThreads = 512;             // cluster and long kernels
constexpr int kChainGridThreads = 256;         // global-memory grid kernels
constexpr uint32_t kChainClusterCap = 65536;   // 16-bit links
constexpr int kChainClusterBatched = 4;        // CTAs per cluster, batched calls
constexpr int kChainClusterSingle = 8;         // CTAs per cluster, one array

// ------------------------------------------------------ index spaces --
__device__ __forceinline__ uint32_t cta_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-bit heads in this CTA's shared memory; the links of positions below
// k_split also, those of higher positions in the CTA's global slot when the
// shared memory is too small for all of them.  Plain loads and stores (the
// passes are ordered by CTA barriers), so the compiler may overlap them.
struct CtaIdx {
    uint16_t *head, *next_s, *next_g;
    uint32_t k_split;
    __device__ __forceinline__ uint16_t *hp(uint32_t y) const { return head + y; }
    __device__ __forceinline__ uint16_t *np(uint32_t c) const {
        return c < k_split ? next_s + c : next_g + (c - k_split);
    }
    // exchange of a 16-bit head; a failed CAS means another push succeeded
    static __device__ __forceinline__ uint32_t exch(uint16_t *a, uint32_t v, uint32_t limit, bool &ok) {
        uint32_t cur = *a;
        for (uint32_t it = 0; it < limit; it++) {
            const uint32_t prev = atomicCAS(reinterpret_cast<unsigned short *>(a), (unsigned short)cur,
                                            (unsigned short)v);
            if (prev == cur) return cur;
            cur = prev;
        }
        ok = false;
        return cur;
    }
    static __device__ __forceinline__ uint32_t ld(const uint16_t *a) { return *a; }
    // pass 3 reads entries other threads are compressing
    static __device__ __forceinline__ uint32_t ld_live(const uint16_t *a) {
        return *reinterpret_cast<const volatile uint16_t *>(a);
    }
    static __device__ __forceinline__ void st(uint16_t *a, uint32_t v) { *a = (uint16_t)v; }
    static __device__ __forceinline__ void st_live(uint16_t *a, uint32_t v) {
        *reinterpret_cast<volatile uint16_t *>(a) = (uint16_t)v;
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
    static __device__ __forceinline__ uint32_t ld_live(uint32_t a) { return ld(a); }
    static __device__ __forceinline__ void st_live(uint32_t a, uint32_t v) { st(a, v); }
};

// 32-bit links in global memory; the head exchanges are atomic (device
// scope).  Loads and stores go through L2 (.cg), which is coherent across the
// SMs at the barriers between passes.
struct GlobalIdx {
    uint32_t *head, *next;
    __device__ __forceinline__ uint32_t *hp(uint32_t y) const { return head + y; }
    __device__ __forceinline__ uint32_t *np(uint32_t c) const { return next + c; }
    static __device__ __forceinline__ uint32_t exch(uint32_t *a, uint32_t v, uint32_t, bool &) {
        return atomicExch(a, v);
    }
    static __device__ __forceinline__ uint32_t ld(const uint32_t *a) { return __ldcg(a); }
    static __device__ __forceinline__ uint32_t ld_live(const uint32_t *a) {
        return *reinterpret_cast<const volatile uint32_t *>(a);
    }
    static __device__ __forceinline__ void st(uint32_t *a, uint32_t v) { __stcg(a, v); }
    static __device__ __forceinline__ void st_live(uint32_t *a, uint32_t v) {
        *reinterpret_cast<volatile uint32_t *>(a) = v;
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

// Pass 2: sort y's list ascending in place, then head[y] <- parent of y (y
// itself when it has none) and the last member's link <- y.  The first
// kSortRegs members are sorted in registers by a sorting network; any
// further ones are linked in by insertion (appended at the tail when larger
// than it, else by a walk of the sorted part).  Only the walker of y
// touches y's members.
constexpr int kSortRegs = 8;

__device__ __forceinline__ void cmp_swap(uint32_t &a, uint32_t &b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

template <class Ix>
__device__ __forceinline__ bool chain_sort(const Ix &ix, uint32_t y, uint32_t limit) {
    const auto hp = ix.hp(y);
    uint32_t m = Ix::ld(hp);
    if (m == 0u) {
        Ix::st(hp, y);
        return true;
    }
    uint32_t v[kSortRegs];
#pragma unroll
    for (int i = 0; i < kSortRegs; i++) {
        v[i] = 0xFFFFFFFFu;  // sorts last
        if (m != 0u) {
            v[i] = m;
            m = Ix::ld(ix.np(m));
        }
    }
    // Batcher-style network for 8 inputs (19 compare-exchanges)
    cmp_swap(v[0], v[1]); cmp_swap(v[2], v[3]); cmp_swap(v[4], v[5]); cmp_swap(v[6], v[7]);
    cmp_swap(v[0], v[2]); cmp_swap(v[1], v[3]); cmp_swap(v[4], v[6]); cmp_swap(v[5], v[7]);
    cmp_swap(v[1], v[2]); cmp_swap(v[5], v[6]); cmp_swap(v[0], v[4]); cmp_swap(v[3], v[7]);
    cmp_swap(v[1], v[5]); cmp_swap(v[2], v[6]); cmp_swap(v[1], v[4]); cmp_swap(v[3], v[6]);
    cmp_swap(v[2], v[4]); cmp_swap(v[3], v[5]); cmp_swap(v[3], v[4]);
    const uint32_t first = v[0];
    uint32_t last = first;
#pragma unroll
    for (int i = 0; i + 1 < kSortRegs; i++) {
        if (v[i + 1] != 0xFFFFFFFFu) {
            Ix::st(ix.np(v[i]), v[i + 1]);
            last = v[i + 1];
        }
    }
    uint32_t head = first;
    uint32_t it = 0;
    while (m != 0u) {  // members beyond the register prefix
        if (++it > limit) return false;
        const auto mp = ix.np(m);
        const uint32_t nx = Ix::ld(mp);  // next unsorted member
        if (m > last) {
            Ix::st(ix.np(last), m);
            last = m;
        } else if (m < head) {
            Ix::st(mp, head);
            head = m;
        } else {
            // head < m < last: the sorted links from head reach a member
            // above m no later than last
            uint32_t p = head;
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
    uint32_t par = head;
    if (head == y) par = head == last ? 0u : Ix::ld(ix.np(head));  // y targets itself
    Ix::st(ix.np(last), y);
    Ix::st(hp, par != 0u ? par : y);
    return true;
}

// Pass 3: head[x] <- root of x.  Any value read is x's parent or a larger
// ancestor (compression only moves entries toward their roots), and a root
// is the only entry equal to its index, so the walk strictly increases.
template <class Ix>
__device__ __forceinline__ bool chain_root(const Ix &ix, uint32_t x, uint32_t limit) {
    const auto qp = ix.hp(x);
    uint32_t r = Ix::ld_live(qp);
    if (r == x) return true;
    for (uint32_t it = 0;; it++) {
        if (it >= limit) return false;
        const uint32_t q = Ix::ld_live(ix.hp(r));
        if (q == r) break;
        r = q;
    }
    Ix::st_live(qp, r);
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

// dst[c] = load(src(c)) for c = start, start + step, ... < end, four at a
// time: all loads of a group are issued before its stores, so a thread has
// four random reads in flight rather than one.
template <typename T, typename SrcFn, typename LoadFn>
__device__ __forceinline__ void gather4(T *dst, uint64_t start, uint64_t step, uint64_t end,
                                        SrcFn srcf, LoadFn load) {
    for (uint64_t c0 = start; c0 < end; c0 += 4 * step) {
        uint32_t src[4];
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint64_t c = c0 + u * step;
            src[u] = c < end ? srcf((uint32_t)c) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (c0 + u * step < end) v[u] = load(src[u]);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint64_t c = c0 + u * step;
            if (c < end) dst[c] = v[u];
        }
    }
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
    uint32_t cta_cap;      // longest array of the CTA kernels (<= 65,536)
    uint32_t cluster_cap;  // up to cluster_cap: one cluster; longer: chain_long_kernel
    uint32_t chunk_cap;    // positions per CTA of the cluster kernel
    uint32_t max_len;
    uint32_t *queue;       // [8]: next array of each kernel (CtaClass::queue, cluster 4, long 5)
    unsigned char *cta_slots;   // large-array CTA kernel: per CTA, a copy of the array, then links
    size_t cta_slot_bytes;
    size_t cta_slot_links;      // offset of the links in a slot
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
// staged whole (eb = 0: heads and links only).
__host__ __device__ __forceinline__ size_t chain_cta_smem(uint32_t n, uint32_t eb) {
    return (((size_t)n * eb + 15) & ~(size_t)15) + 2 * (((size_t)n + 7) & ~(size_t)7) * 2;
}

// A size class of the CTA kernel: arrays with lo < n <= hi, one CTA each.
struct CtaClass {
    uint32_t lo, hi;
    uint32_t full_cap;    // staged whole (elements, heads, links) up to this length
    uint32_t link_bytes;  // shared memory for the heads and links of longer arrays
    uint32_t queue;       // index of the class's work counter
    uint32_t validate;    // record BRR_EINVAL for invalid arrays
};

// One CTA per array at a time, in a size class.  Arrays up to full_cap are
// staged whole in shared memory.  Longer ones keep their heads (the random
// atomics of pass 1, the parent forest of passes 3-4) and as many links as
// fit in shared memory; the element copy and the remaining links go to the
// CTA's global slot, which stays resident in L2 while the CTA works on it.
// Small classes use small CTAs, so that several arrays are in flight per SM
// and their fixed latencies (queue, plan, barriers) overlap.
template <typename T, int kThreads>
__global__ void __launch_bounds__(kThreads) chain_cta_kernel(ChainArgs a, CtaClass cls) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ChainCtl ctl;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) ctl.err = 0;
    const uint32_t n_items = a.offsets ? a.n_arrays : 1u;
    for (;;) {
        __syncthreads();
        if (tid == 0) ctl.item[0] = atomicAdd(&a.queue[cls.queue], 1u);
        __syncthreads();
        const uint32_t s = ctl.item[0];
        if (s >= n_items) break;
        uint64_t o0, len, seed;
        if (!chain_item(a, s, o0, len, seed)) {
            if (cls.validate && tid == 0) ctl.err = BRR_EINVAL;
            continue;
        }
        if (len < 2 || len <= cls.lo || len > cls.hi) continue;
        const uint32_t n = (uint32_t)len;
        if (tid == 0) chain_plan(ctl, a, n);
        T *g = static_cast<T *>(a.data) + o0;
        const uint32_t n8 = (n + 7) & ~7u;
        const bool staged = n <= cls.full_cap;
        unsigned char *slot = a.cta_slots + (size_t)blockIdx.x * a.cta_slot_bytes;
        T *As;
        uint16_t *head;
        uint32_t k_split = n;
        if (staged) {
            As = reinterpret_cast<T *>(smem);
            head = reinterpret_cast<uint16_t *>(smem + (((size_t)n * sizeof(T) + 15) & ~(size_t)15));
        } else {
            As = reinterpret_cast<T *>(slot);
            head = reinterpret_cast<uint16_t *>(smem);
            k_split = min(n, (cls.link_bytes / 2 - n8) & ~7u);
        }
        const CtaIdx ix{head, head + n8, reinterpret_cast<uint16_t *>(slot + a.cta_slot_links), k_split};
        gather4(As, tid, kThreads, n, [](uint32_t x) { return x; }, [&](uint32_t x) { return g[x]; });
        for (uint32_t x = tid; x < n; x += kThreads) {
            head[x] = 0;
            *ix.np(x) = 0;
        }
        __syncthreads();
        if (ctl.nseg == 0) continue;
        const uint32_t lim = chain_limit(n);
        uint32_t *jo = a.j_out;
        bool ok = true;
        roll_plan_range(ctl.seg, ctl.nseg, 0, ctl.n_batches, seed, ctl.err, [&](uint32_t pos, uint32_t v) {
            if (jo) jo[pos] = v;
            ok = chain_push(ix, pos, v, lim) && ok;
        });
        if (jo && tid == 0) jo[0] = 0;
        __syncthreads();
        for (uint32_t y = tid; y < n; y += kThreads) ok = chain_sort(ix, y, lim) && ok;
        __syncthreads();
        for (int32_t x = (int32_t)n - 1 - (int32_t)tid; x >= 0; x -= kThreads)
            ok = chain_root(ix, (uint32_t)x, lim) && ok;
        __syncthreads();
        gather4(g, tid, kThreads, n, [&](uint32_t c) { return chain_source(ix, c); },
                [&](uint32_t x) { return As[x]; });
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
        if (rank == 0 && tid == 0) ctl.item[par] = atomicAdd(&a.queue[4], 1u);
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
        if (tid == 0) ctl.item[0] = atomicAdd(&a.queue[5], 1u);
        __syncthreads();
        const uint32_t s = ctl.item[0];
        if (s >= n_items) break;
        uint64_t o0, len, seed;
        if (!chain_item(a, s, o0, len, seed)) continue;  // reported by the CTA kernel
        if (len <= a.cluster_cap) continue;
        const uint32_t n = (uint32_t)len;
        if (tid == 0) chain_plan(ctl, a, n);
        T *g = static_cast<T *>(a.data) + o0;
        gather4(copy, tid, blockDim.x, n, [](uint32_t x) { return x; }, [&](uint32_t x) { return g[x]; });
        for (uint32_t x = tid; x < n; x += blockDim.x) {
            head[x] = 0;
            next[x] = 0;
        }
        __syncthreads();
        if (ctl.nseg == 0) continue;
        const GlobalIdx ix{head, next};
        const uint32_t lim = chain_limit(n);
        bool ok = true;
        roll_plan_range(ctl.seg, ctl.nseg, 0, ctl.n_batches, seed, ctl.err,
                        [&](uint32_t pos, uint32_t v) { ok = chain_push(ix, pos, v, lim) && ok; });
        __syncthreads();
        for (uint32_t y = tid; y < n; y += blockDim.x) ok = chain_sort(ix, y, lim) && ok;
        __syncthreads();
        for (int64_t x = (int64_t)n - 1 - tid; x >= 0; x -= blockDim.x) ok = chain_root(ix, (uint32_t)x, lim) && ok;
        __syncthreads();
        gather4(g, tid, blockDim.x, n, [&](uint32_t c) { return chain_source(ix, c); },
                [&](uint32_t x) { return __ldcg(&copy[x]); });
        if (!ok) ctl.err = BRR_ETIMEOUT;
    }
    __syncthreads();
    if (tid == 0 && ctl.err) record_error(a.err, ctl.err);
}

// ------------------------------------------------- one array, whole grid --
// One cooperative launch: clear the links and copy the array, push, sort,
// root, gather -- grid-stride loops separated by bounded grid barriers.  If
// a barrier gives up (or any error is recorded) every block leaves before
// the gather, so the array is left as it was.
struct ChainGridArgs {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
    uint64_t seed;
    uint32_t *head, *next;
    void *data, *copy;
    uint32_t n;
    uint32_t *j_out;
    uint32_t *bar;  // [2] grid barrier, zero on entry
    int *err;
};

// The phases, each a grid-stride loop over the launch's threads.  They run
// in one cooperative launch separated by grid barriers (lowest latency), or
// as one launch each (no co-residency needed, so they share the GPU with
// kernels on other streams).
template <typename T>
__device__ __forceinline__ void grid_phase(const ChainGridArgs &a, int phase, uint64_t gid, uint64_t stride) {
    const GlobalIdx ix{a.head, a.next};
    const uint32_t lim = chain_limit(a.n);
    T *A = static_cast<T *>(a.data);
    T *copy = static_cast<T *>(a.copy);
    bool ok = true;
    if (phase == 0) {
        gather4(copy, gid, stride, a.n, [](uint32_t x) { return x; }, [&](uint32_t x) { return A[x]; });
        for (uint64_t x = gid; x < a.n; x += stride) {
            a.head[x] = 0;
            a.next[x] = 0;
        }
    } else if (phase == 1) {
        bool rolled = true;
        for (uint64_t g = gid; g < a.n_batches; g += stride)
            rolled = roll_plan_batch(a.seg, a.nseg, g, a.seed, [&](uint32_t pos, uint32_t v) {
                         if (a.j_out) a.j_out[pos] = v;
                         ok = chain_push(ix, pos, v, lim) && ok;
                     }) && rolled;
        if (a.j_out && gid == 0) a.j_out[0] = 0;
        if (!rolled) record_error(a.err, BRR_ERETRY);
    } else if (phase == 2) {
        for (uint64_t y = gid; y < a.n; y += stride)
            if (!chain_sort(ix, (uint32_t)y, lim)) ok = false;
    } else if (phase == 3) {
        for (int64_t x = (int64_t)a.n - 1 - (int64_t)gid; x >= 0; x -= (int64_t)stride)
            if (!chain_root(ix, (uint32_t)x, lim)) ok = false;
    } else {
        gather4(A, gid, stride, a.n, [&](uint32_t c) { return chain_source(ix, c); },
                [&](uint32_t x) { return __ldcg(&copy[x]); });
    }
    if (!ok) record_error(a.err, BRR_ETIMEOUT);
}

template <typename T>
__global__ void __launch_bounds__(kChainGridThreads) chain_grid_kernel(ChainGridArgs a) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int phase = 0; phase < 5; phase++) {
        if (phase > 0 && !grid_barrier(a.bar, a.err)) return;
        grid_phase<T>(a, phase, gid, stride);
    }
}

// One phase per launch.  The gather is skipped once an error is recorded
// (the array is then left as it was).
template <typename T>
__global__ void __launch_bounds__(kChainGridThreads) chain_grid_phase_kernel(ChainGridArgs a, int phase) {
    if (phase == 4 && ld_relaxed_i32(a.err) != 0) return;
    grid_phase<T>(a, phase, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
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

// Kernel attributes and occupancy, once per context and element size (and
// again after brr_tune changes a class boundary).  Classes: 0 small (128
// threads), 1 medium (256), 2 large (1024, all of the shared memory).
constexpr int kClassThreads[3] = {128, 256, 1024};

template <typename T>
static const void *cta_kernel_of(int cls) {
    return cls == 0 ? (const void *)chain_cta_kernel<T, 128>
                    : cls == 1 ? (const void *)chain_cta_kernel<T, 256> : (const void *)chain_cta_kernel<T, 1024>;
}

template <typename T>
static brr_status chain_setup(brr_ctx *ctx) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    if (ctx->chain_ready[ix]) return BRR_OK;
    const size_t limit = ((size_t)ctx->max_smem_optin - sizeof(ChainCtl) - 1024) & ~(size_t)15;
    uint32_t full = (uint32_t)std::min<size_t>(limit / (sizeof(T) + 4), kChainClusterCap);
    while (full > 0 && chain_cta_smem(full, sizeof(T)) > limit) full--;
    const uint32_t hi_l = (uint32_t)std::min<size_t>((limit / 2) & ~(size_t)7, kChainClusterCap);
    const uint32_t hi_s = (uint32_t)std::min<uint64_t>(ctx->tune.small_max, full);
    const uint32_t hi_m = std::max(hi_s, (uint32_t)std::min<uint64_t>(ctx->tune.medium_max, full));
    uint32_t link_cap = (uint32_t)std::min<size_t>(limit / 4, kChainClusterCap);
    while (link_cap > 0 && chain_cta_smem(link_cap, 0) > limit) link_cap--;
    brr_ctx::ChainClass cls[3];
    cls[0] = {0, hi_s, hi_s, 0, hi_s, chain_cta_smem(hi_s, sizeof(T)), 0};
    cls[1] = {hi_s, hi_m, hi_m, 0, hi_m, chain_cta_smem(hi_m, sizeof(T)), 0};
    cls[2] = {hi_m, std::max(hi_m, hi_l), full, (uint32_t)limit, link_cap, limit, 0};
    for (int c = 0; c < 3; c++) {
        const void *k = cta_kernel_of<T>(c);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cls[c].smem);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cls[c].per_sm, k, kClassThreads[c], cls[c].smem);
        if (e != cudaSuccess || cls[c].per_sm < 1) return BRR_ECUDA;
        ctx->chain_cls[ix][c] = cls[c];
    }
    int long_per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&long_per_sm, chain_long_kernel<T>, kChainThreads, 0);
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
    ctx->chain_long_per_sm[ix] = long_per_sm;
    ctx->chain_clusters[ix][0] = clusters[0];
    ctx->chain_clusters[ix][1] = clusters[1];
    ctx->chain_ready[ix] = true;
    return BRR_OK;
}

// One CTA-kernel launch of class c; `single` (one array) takes any length up
// to the class's limit.
template <typename T>
static cudaError_t launch_cta_class(brr_ctx *ctx, int c, const ChainArgs &a, uint32_t grid,
                                    bool validate, bool single, cudaStream_t stream) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    const brr_ctx::ChainClass &k = ctx->chain_cls[ix][c];
    const CtaClass cls = {single ? 0u : k.lo, std::min(k.hi, a.cta_cap), k.full_cap, k.link_bytes,
                          (uint32_t)c, validate ? 1u : 0u};
    if (c == 0) chain_cta_kernel<T, 128><<<grid, 128, k.smem, stream>>>(a, cls);
    else if (c == 1) chain_cta_kernel<T, 256><<<grid, 256, k.smem, stream>>>(a, cls);
    else chain_cta_kernel<T, 1024><<<grid, 1024, k.smem, stream>>>(a, cls);
    return cudaGetLastError();
}

// Batched shuffles (offsets != nullptr), or one array (offsets == nullptr)
// of at most kChainClusterCap elements.  Which kernel takes an array:
//   batched: n <= small/medium/large class limit   chain_cta_kernel of that class
//            n <= 65,536, tune.batched_cluster = 1: chain_cluster_kernel, 4 CTAs
//            longer                                chain_long_kernel
//   one:     single_cta: the large-class CTA kernel; otherwise a cluster of 8
template <typename T>
static brr_status launch_chains_staged(brr_ctx *ctx, ChainArgs a, uint64_t max_len, bool single_cta,
                                       cudaStream_t stream) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    brr_status st = chain_setup<T>(ctx);
    if (st != BRR_OK) return st;
    const brr_ctx::ChainClass *cls = ctx->chain_cls[ix];
    const bool single = a.offsets == nullptr;
    const uint32_t n_items = single ? 1u : a.n_arrays;
    a.max_len = (uint32_t)max_len;
    a.err = ctx->d_err;
    // with batched clusters on, arrays whose links do not fit go to them
    a.cta_cap = (!single && ctx->tune.batched_cluster) ? std::min(cls[2].link_cap, cls[2].hi) : cls[2].hi;
    const bool use_cluster = single ? !single_cta : (ctx->tune.batched_cluster != 0 && max_len > a.cta_cap);
    a.cluster_cap = single ? kChainClusterCap : (ctx->tune.batched_cluster ? kChainClusterCap : a.cta_cap);
    const uint32_t csize = single ? kChainClusterSingle : kChainClusterBatched;
    a.chunk_cap = kChainClusterCap / csize;
    bool run[3];
    uint32_t grid[3];
    for (int c = 0; c < 3; c++) {
        run[c] = single ? (single_cta && c == 2) : (c == 0 || max_len > cls[c].lo);
        grid[c] = (uint32_t)std::min<uint64_t>((uint64_t)cls[c].per_sm * ctx->num_sms, n_items);
    }
    // global slots of the large class (element copies and the links that do
    // not fit), and of the long kernel (links and copies)
    size_t cta_slots = 0;
    if (run[2] && max_len > cls[2].full_cap) {
        const uint64_t most = std::min<uint64_t>(max_len, a.cta_cap);
        a.cta_slot_links = ((size_t)most * sizeof(T) + 255) & ~(size_t)255;
        a.cta_slot_bytes = a.cta_slot_links + (((size_t)most * 2 + 255) & ~(size_t)255);
        cta_slots = (size_t)grid[2] * a.cta_slot_bytes;
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
    cudaError_t e = cudaMemsetAsync(a.queue, 0, 8 * sizeof(uint32_t), stream);
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
    // large arrays first; the small class also validates every array
    for (int c = 2; c >= 0; c--) {
        if (!run[c]) continue;
        e = launch_cta_class<T>(ctx, c, a, grid[c], c == 0 || single, single, stream);
        if (e != cudaSuccess) return cuda_status(e);
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

// Resident blocks per SM of the grid kernel (the cooperative launch needs
// every block resident), queried once per process and element size.
static int chain_grid_per_sm(uint32_t elem_bytes) {
    static int cached[2] = {0, 0};
    int &c = cached[elem_bytes == 4 ? 0 : 1];
    if (c == 0) {
        int v = 0;
        const cudaError_t e = elem_bytes == 4
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, chain_grid_kernel<uint32_t>, kChainGridThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, chain_grid_kernel<uint64_t>, kChainGridThreads, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        c = v;
    }
    return c;
}

// One array of up to 2^32 - 2 elements on `scratch` (chains_grid_scratch
// bytes: barrier words, heads, links and a copy of the array), in one
// cooperative launch or in five launches.
brr_status launch_chains_grid(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                              const brr_schedule *sched, uint32_t *j_out, void *scratch, int *err,
                              int num_sms, cudaStream_t stream, bool cooperative) {
    ChainGridArgs a;
    a.nseg = plan_segments(n, 1, sched->n_k, sched->k_max, a.seg, kMaxSegs, &a.n_batches);
    if (a.nseg < 0) return BRR_EINVAL;
    a.seed = seed;
    a.n = (uint32_t)n;
    a.j_out = j_out;
    a.err = err;
    a.data = data;
    const size_t links = ((size_t)n * 4 + 255) & ~(size_t)255;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    a.bar = reinterpret_cast<uint32_t *>(base);
    a.head = reinterpret_cast<uint32_t *>(base + 256);
    a.next = reinterpret_cast<uint32_t *>(base + 256 + links);
    a.copy = base + 256 + 2 * links;
    const int per_sm = chain_grid_per_sm(elem_bytes);
    if (per_sm < 1) return BRR_ECUDA;
    // enough blocks for one position (or batch) per thread, at most all resident
    const uint64_t want = (std::max<uint64_t>(n, a.n_batches) + kChainGridThreads - 1) / kChainGridThreads;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)per_sm * num_sms));
    cudaError_t e;
    if (!cooperative) {
        const uint64_t cap = (uint64_t)per_sm * num_sms;
        for (int phase = 0; phase < 5; phase++) {
            const uint64_t units = phase == 1 ? a.n_batches : n;
            const unsigned g = (unsigned)std::max<uint64_t>(
                1, std::min<uint64_t>(cap, (units + kChainGridThreads - 1) / kChainGridThreads));
            if (elem_bytes == 4)
                chain_grid_phase_kernel<uint32_t><<<g, kChainGridThreads, 0, stream>>>(a, phase);
            else
                chain_grid_phase_kernel<uint64_t><<<g, kChainGridThreads, 0, stream>>>(a, phase);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
        }
        return BRR_OK;
    }
    e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    void *args[] = {&a};
    e = elem_bytes == 4
        ? cudaLaunchCooperativeKernel((const void *)chain_grid_kernel<uint32_t>, grid, kChainGridThreads, args, 0, stream)
        : cudaLaunchCooperativeKernel((const void *)chain_grid_kernel<uint64_t>, grid, kChainGridThreads, args, 0, stream);
    return cuda_status(e);
}

// One array: one CTA up to tune.single_cta_max elements, one cluster of 8
// up to tune.single_cluster_max (at most 65,536), else the grid passes.
brr_status launch_chains_one(brr_ctx *ctx, void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                             const brr_schedule *sched, uint32_t *j_out, cudaStream_t stream) {
    const int ix = elem_bytes == 4 ? 0 : 1;
    brr_status st = elem_bytes == 4 ? chain_setup<uint32_t>(ctx) : chain_setup<uint64_t>(ctx);
    if (st != BRR_OK) return st;
    const bool cta = n <= std::min<uint64_t>(ctx->tune.single_cta_max, ctx->chain_cls[ix][2].hi);
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
                              ctx->num_sms, stream, ctx->tune.grid_cooperative != 0);
}

}  // namespace brr
