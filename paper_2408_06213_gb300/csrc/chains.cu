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
// A step with j_c = c is the smallest possible member of its own group, so
// succ(c) = parent(c) and final[c] = A[W(c)]; such steps are kept out of the
// lists and their link records "c".
//
// Passes (each fully parallel, separated by a barrier):
//  1. roll every batch of the plan (Algorithm 4) and push step c onto the
//     list of target y = j_c with one atomic exchange of the list head.  The
//     old head becomes c's link; on an empty list the link is y itself (a
//     link <= its position then always means "no successor, the target is
//     the link").  Steps are pushed in nearly decreasing order, so a list
//     read from its head is nearly ascending: a push that finds a smaller
//     head (out of order) flags the list in a bitmap.
//  2. per target y: an empty list gives parent(y) = none; an unflagged list
//     is ascending with its last link already y, so its head is parent(y)
//     and nothing is written; a flagged list is sorted in place.
//  3. per x, in decreasing order: replace parent(x) by the root (path
//     compression; parents are larger, so they are mostly finished already).
//  4. per position c: gather final[c] from the original array.
//
// Tiers share the passes through an index-space accessor: one CTA with 16-bit
// links in its shared memory (arrays of up to 65,536 elements, in three size
// classes), and global memory with 32-bit links in scratch (one CTA per
// array, or the whole grid).  Every loop is bounded by the array length; a
// bound that runs out records BRR_ETIMEOUT instead of looping.
#include <algorithm>
#include <type_traits>

#include "brr_common.cuh"
#include "internal.h"
#include "words.cuh"

namespace brr {

constexpr int kChainThreads = 512;             // long-array kernel
constexpr int kChainGridThreads = 256;         // grid-wide kernels
constexpr uint32_t kChainCtaCap = 65536;       // 16-bit links
constexpr uint32_t kChainBinClasses = 9;       // size-class lists: 0-2 CTA classes, 3 long, 4-8 windows
constexpr uint32_t kChainBinMaxArrays = 1u << 24;  // calls with more arrays go without lists
constexpr uint32_t kWinSmallMax = 4096;        // the windows take the small class up to this limit

// ------------------------------------------------------ index spaces --
// 16-bit heads and the out-of-order bitmap in this CTA's shared memory; the
// links of positions below k_split also, those of higher positions in the
// CTA's global slot when the shared memory is too small for all of them.
// Plain loads and stores (the passes are ordered by CTA barriers), so the
// compiler may overlap them.
struct CtaIdx {
    uint16_t *head, *next_s, *next_g;
    uint32_t *bits;
    uint32_t k_split;
    __device__ __forceinline__ uint16_t *hp(uint32_t y) const { return head + y; }
    __device__ __forceinline__ uint16_t *np(uint32_t c) const {
        return c < k_split ? next_s + c : next_g + (c - k_split);
    }
    __device__ __forceinline__ void mark(uint32_t y) const { atomicOr(&bits[y >> 5], 1u << (y & 31u)); }
    __device__ __forceinline__ bool marked(uint32_t y) const { return (bits[y >> 5] >> (y & 31u)) & 1u; }
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

// The same with every link in shared memory (arrays staged whole): every
// access is a plain shared-memory one, with no per-access choice of space.
struct CtaIdxS {
    uint16_t *head, *next_s;
    uint32_t *bits;
    __device__ __forceinline__ uint16_t *hp(uint32_t y) const { return head + y; }
    __device__ __forceinline__ uint16_t *np(uint32_t c) const { return next_s + c; }
    __device__ __forceinline__ void mark(uint32_t y) const { atomicOr(&bits[y >> 5], 1u << (y & 31u)); }
    __device__ __forceinline__ bool marked(uint32_t y) const { return (bits[y >> 5] >> (y & 31u)) & 1u; }
    static __device__ __forceinline__ uint32_t exch(uint16_t *a, uint32_t v, uint32_t limit, bool &ok) {
        return CtaIdx::exch(a, v, limit, ok);
    }
    static __device__ __forceinline__ uint32_t ld(const uint16_t *a) { return *a; }
    static __device__ __forceinline__ uint32_t ld_live(const uint16_t *a) {
        return *reinterpret_cast<const volatile uint16_t *>(a);
    }
    static __device__ __forceinline__ void st(uint16_t *a, uint32_t v) { *a = (uint16_t)v; }
    static __device__ __forceinline__ void st_live(uint16_t *a, uint32_t v) {
        *reinterpret_cast<volatile uint16_t *>(a) = (uint16_t)v;
    }
};

// 32-bit heads, links and bitmap in global memory; the head exchanges are
// atomic (device scope).  Loads and stores go through L2 (.cg), which is
// coherent across the SMs at the barriers between passes.
struct GlobalIdx {
    uint32_t *head, *next, *bits;
    __device__ __forceinline__ uint32_t *hp(uint32_t y) const { return head + y; }
    __device__ __forceinline__ uint32_t *np(uint32_t c) const { return next + c; }
    __device__ __forceinline__ void mark(uint32_t y) const { atomicOr(&bits[y >> 5], 1u << (y & 31u)); }
    __device__ __forceinline__ bool marked(uint32_t y) const { return (__ldcg(&bits[y >> 5]) >> (y & 31u)) & 1u; }
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
// Pass 1: step c (1 <= c < n) with target y <= c.
template <class Ix>
__device__ __forceinline__ bool chain_push(const Ix &ix, uint32_t c, uint32_t y, uint32_t limit) {
    if (y == c) {
        Ix::st(ix.np(c), c);
        return true;
    }
    bool ok = true;
    const uint32_t old = Ix::exch(ix.hp(y), c, limit, ok);
    Ix::st(ix.np(c), old != 0u ? old : y);
    if (old != 0u && old < c) ix.mark(y);
    return ok;
}

// Pass 2 for a flagged list: sort it ascending in place.  Members are linked
// in by insertion (appended at the tail when larger than it, else by a walk
// of the sorted part); the unsorted list ends at the member whose link is y
// (members are all above y).  kNetwork first gathers up to kSortRegs members
// into registers and sorts them with a bitonic network, for lists pushed in
// random order: the pass then costs one chain of dependent loads per list
// rather than a walk of the sorted part for every member.
constexpr int kSortRegs = 16;

__device__ __forceinline__ void cmp_swap(uint32_t &a, uint32_t &b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Sorts the list's first kSortRegs members (head, then from m on until the
// end marker y) in registers and links them; returns the next unsorted
// member (or y).
template <class Ix>
__device__ __forceinline__ uint32_t sort_prefix(const Ix &ix, uint32_t y, uint32_t &head, uint32_t &last,
                                                uint32_t m) {
    uint32_t v[kSortRegs];
    v[0] = head;
#pragma unroll
    for (int i = 1; i < kSortRegs; i++) {
        v[i] = 0xFFFFFFFFu;  // sorts last
        if (m != y) {
            v[i] = m;
            m = Ix::ld(ix.np(m));
        }
    }
    // bitonic network over kSortRegs (a power of two) inputs, ascending
#pragma unroll
    for (int kk = 2; kk <= kSortRegs; kk <<= 1) {
#pragma unroll
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
#pragma unroll
            for (int i = 0; i < kSortRegs; i++) {
                const int l = i ^ jj;
                if (l > i) {
                    if ((i & kk) == 0) cmp_swap(v[i], v[l]);
                    else cmp_swap(v[l], v[i]);
                }
            }
        }
    }
    head = last = v[0];
#pragma unroll
    for (int i = 0; i + 1 < kSortRegs; i++) {
        if (v[i + 1] != 0xFFFFFFFFu) {
            Ix::st(ix.np(v[i]), v[i + 1]);
            last = v[i + 1];
        }
    }
    return m;
}

// Pass 2: head[y] <- parent of y (y itself when it has none).
template <bool kNetwork, class Ix>
__device__ __forceinline__ bool chain_fix(const Ix &ix, uint32_t y, uint32_t limit) {
    const auto hp = ix.hp(y);
    const uint32_t h = Ix::ld(hp);
    if (h == 0u) {
        Ix::st(hp, y);
        return true;
    }
    if (!ix.marked(y)) return true;  // ascending already; the head is the parent
    uint32_t head = h, last = h;      // the sorted part so far: the first member
    uint32_t m = Ix::ld(ix.np(h));
    if (kNetwork) m = sort_prefix(ix, y, head, last, m);
    uint32_t it = 0;
    while (m != y) {
        if (++it > limit) return false;
        const auto mp = ix.np(m);
        const uint32_t nx = Ix::ld(mp);  // next unsorted member, or y
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
    Ix::st(ix.np(last), y);
    Ix::st(hp, head);
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
    return l >= c ? Ix::ld(ix.hp(l)) : l;
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
    uint32_t item;
};

struct ChainArgs {
    void *data;
    const uint64_t *offsets;  // nullptr: one array of single_n elements
    const uint64_t *seeds;
    uint32_t n_arrays;
    uint64_t nk[BRR_SCHED_KMAX + 1];
    uint32_t k_max;
    uint32_t max_len;
    uint32_t *queue;            // [8]: next array of each kernel (CtaClass::queue; long kernel 3)
    unsigned char *cta_slots;   // large-class CTA kernel: per CTA, a copy of the array, then links
    size_t cta_slot_bytes;
    size_t cta_slot_links;      // offset of the links in a slot
    unsigned char *slots;       // long kernel: per CTA, heads, links, bitmap and a copy
    size_t slot_bytes;
    uint32_t single_n;
    uint64_t single_seed;
    uint32_t *j_out;            // single-array form: swap indices (optional)
    uint32_t ordered_push;      // CTA kernel: a barrier between rounds of batch rolls
    const uint32_t *bin_list;   // batched arrays sorted by size class: [class][n_arrays] (null: none)
    const uint32_t *bin_count;  //   and how many each class has
    int *err;
};

// Work item i of a size-class kernel (class c, work counter c): the i-th
// array of the class's list, or array i itself without lists.  Returns false
// past the end.
__device__ __forceinline__ bool chain_next(const ChainArgs &a, uint32_t c, uint32_t i, uint32_t &s) {
    if (a.bin_list) {
        if (i >= a.bin_count[c]) return false;
        s = a.bin_list[(size_t)c * a.n_arrays + i];
        return true;
    }
    s = i;
    return i < (a.offsets ? a.n_arrays : 1u);
}

// Sorts the batched arrays into the lists of the size classes (one thread per
// array): class c takes the lengths len with bound[c-1] < len <= bound[c]
// (len >= 2; shorter arrays need no work).  Invalid arrays (offsets that
// decrease, lengths above max_len) record BRR_EINVAL here.
struct ChainBins {
    uint32_t n_cls;
    uint64_t bound[8];
    uint32_t cls[8];
};

__global__ void chain_bin_kernel(const uint64_t *offsets, uint32_t n_arrays, uint64_t max_len, ChainBins b,
                                 uint32_t *list, uint32_t *count, int *err) {
    int e = 0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_arrays; s += gridDim.x * blockDim.x) {
        const uint64_t o0 = offsets[s], o1 = offsets[s + 1];
        if (o1 < o0 || o1 - o0 > max_len) {
            e = BRR_EINVAL;
            continue;
        }
        const uint64_t len = o1 - o0;
        if (len < 2) continue;
        uint32_t c = b.cls[b.n_cls - 1];
        for (uint32_t i = 0; i + 1 < b.n_cls; i++) {
            if (len <= b.bound[i]) {
                c = b.cls[i];
                break;
            }
        }
        list[(size_t)c * n_arrays + atomicAdd(&count[c], 1u)] = s;
    }
    if (e) record_error(err, e);
}

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

// Shared-memory layout of the CTA kernel for an array of n elements of eb
// bytes: the elements when staged (eb = 0: not staged), the heads, the
// out-of-order bitmap, then the links held in shared memory.
struct CtaLayout {
    size_t head, bits, next;
    __host__ __device__ CtaLayout(uint32_t n, uint32_t eb) {
        head = ((size_t)n * eb + 15) & ~(size_t)15;
        bits = head + (((size_t)n + 7) & ~(size_t)7) * 2;
        next = bits + ((((size_t)n + 31) / 32 * 4 + 15) & ~(size_t)15);
    }
    __host__ __device__ size_t staged_bytes(uint32_t n) const { return next + (((size_t)n + 7) & ~(size_t)7) * 2; }
};

// A size class of the CTA kernel: arrays with lo < n <= hi, one CTA each.
struct CtaClass {
    uint32_t lo, hi;
    uint32_t full_cap;    // staged whole (elements, heads, links) up to this length
    uint32_t link_bytes;  // shared memory for heads, bitmap and links of longer arrays
    uint32_t queue;       // index of the class's work counter
    uint32_t validate;    // record BRR_EINVAL for invalid arrays
};

// One CTA per array at a time, in a size class.  Arrays up to full_cap are
// staged whole in shared memory.  Longer ones keep their heads (the random
// atomics of pass 1, the parent forest of passes 3-4), the bitmap and as
// many links as fit in shared memory; the element copy and the remaining
// links go to the CTA's global slot, which stays resident in L2 while the
// CTA works on it.  Small classes use small CTAs, so that several arrays are
// in flight per SM and their fixed latencies (queue, plan, barriers) overlap.
template <typename T, int kThreads, uint32_t SRC = BRR_WORDS_SPLITMIX64, bool kStagedOnly = false>
__global__ void __launch_bounds__(kThreads) chain_cta_kernel(ChainArgs a, CtaClass cls) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ChainCtl ctl;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) ctl.err = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) ctl.item = atomicAdd(&a.queue[cls.queue], 1u);
        __syncthreads();
        uint32_t s;
        if (!chain_next(a, cls.queue, ctl.item, s)) break;
        uint64_t o0, len, seed;
        if (!chain_item(a, s, o0, len, seed)) {
            if (cls.validate && tid == 0) ctl.err = BRR_EINVAL;
            continue;
        }
        if (len < 2 || len <= cls.lo || len > cls.hi) continue;
        const uint32_t n = (uint32_t)len;
        if (tid == 0) chain_plan(ctl, a, n);
        T *g = static_cast<T *>(a.data) + o0;
        // kStagedOnly (every array of the class fits): elements, heads,
        // bitmap and links in shared memory, all accesses shared-memory ones.
        // Otherwise arrays above full_cap keep the element copy and the links
        // above k_split in the CTA's L2 slot, and the index space chooses the
        // space per link.
        const bool staged = kStagedOnly || n <= cls.full_cap;
        const CtaLayout lay(n, staged ? (uint32_t)sizeof(T) : 0u);
        unsigned char *slot = a.cta_slots + (size_t)blockIdx.x * a.cta_slot_bytes;
        T *As = staged ? reinterpret_cast<T *>(smem) : reinterpret_cast<T *>(slot);
        uint32_t k_split = n;
        if (!staged) k_split = min(n, (uint32_t)((cls.link_bytes - lay.next) / 2) & ~7u);
        using Ix = typename std::conditional<kStagedOnly, CtaIdxS, CtaIdx>::type;
        Ix ix;
        if constexpr (kStagedOnly) {
            ix = CtaIdxS{reinterpret_cast<uint16_t *>(smem + lay.head), reinterpret_cast<uint16_t *>(smem + lay.next),
                         reinterpret_cast<uint32_t *>(smem + lay.bits)};
        } else {
            ix = CtaIdx{reinterpret_cast<uint16_t *>(smem + lay.head), reinterpret_cast<uint16_t *>(smem + lay.next),
                        reinterpret_cast<uint16_t *>(slot + a.cta_slot_links),
                        reinterpret_cast<uint32_t *>(smem + lay.bits), k_split};
        }
        gather4(As, tid, kThreads, n, [](uint32_t x) { return x; }, [&](uint32_t x) { return g[x]; });
        for (uint32_t x = tid; x < n; x += kThreads) ix.head[x] = 0;
        for (uint32_t w = tid; w < (n + 31) / 32; w += kThreads) ix.bits[w] = 0;
        __syncthreads();
        if (ctl.nseg == 0) continue;
        const uint32_t lim = chain_limit(n);
        uint32_t *jo = a.j_out;
        bool ok = true;
        auto push = [&](uint32_t pos, uint32_t v) {
            if (jo) jo[pos] = v;
            ok = chain_push(ix, pos, v, lim) && ok;
        };
        if (a.ordered_push) {
            // rounds of kThreads batches, largest positions first, with a
            // barrier between rounds: a list's pushes from different rounds
            // then arrive in sequential (decreasing) order, and only pushes
            // of one round to one target can be out of order
            for (uint64_t base = 0; base < ctl.n_batches; base += kThreads) {
                const uint64_t gb = base + tid;
                if (gb < ctl.n_batches && !roll_plan_batch_src<SRC>(ctl.seg, ctl.nseg, gb, seed, push))
                    ctl.err = BRR_ERETRY;
                __syncthreads();
            }
        } else {
            roll_plan_range_src<SRC>(ctl.seg, ctl.nseg, 0, ctl.n_batches, seed, ctl.err, push);
        }
        if (jo && tid == 0) jo[0] = 0;
        __syncthreads();
        for (uint32_t y = tid; y < n; y += kThreads) ok = chain_fix<false>(ix, y, lim) && ok;
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

// Layout of one long-kernel slot: heads, links, bitmap (32-bit) and a copy
// of the array, for arrays of up to max_len elements.
struct SlotLayout {
    size_t next, bits, copy, bytes;
    __host__ __device__ SlotLayout(uint64_t max_len, uint32_t eb) {
        const size_t links = ((size_t)max_len * 4 + 255) & ~(size_t)255;
        next = links;
        bits = 2 * links;
        copy = bits + ((((size_t)max_len + 31) / 32 * 4 + 255) & ~(size_t)255);
        bytes = copy + (((size_t)max_len * eb + 255) & ~(size_t)255);
    }
};

// Batched arrays longer than 65,536 elements: one CTA per array in global
// memory, with scratch slot blockIdx.x (resident in L2 while it is used).
template <typename T, uint32_t SRC = BRR_WORDS_SPLITMIX64>
__global__ void __launch_bounds__(kChainThreads) chain_long_kernel(ChainArgs a) {
    __shared__ ChainCtl ctl;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) ctl.err = 0;
    const SlotLayout lay(a.max_len, sizeof(T));
    unsigned char *slot = a.slots + (size_t)blockIdx.x * a.slot_bytes;
    const GlobalIdx ix{reinterpret_cast<uint32_t *>(slot), reinterpret_cast<uint32_t *>(slot + lay.next),
                       reinterpret_cast<uint32_t *>(slot + lay.bits)};
    T *copy = reinterpret_cast<T *>(slot + lay.copy);
    for (;;) {
        __syncthreads();
        if (tid == 0) ctl.item = atomicAdd(&a.queue[3], 1u);
        __syncthreads();
        uint32_t s;
        if (!chain_next(a, 3, ctl.item, s)) break;
        uint64_t o0, len, seed;
        if (!chain_item(a, s, o0, len, seed)) continue;  // reported by the CTA kernel
        if (len <= kChainCtaCap) continue;
        const uint32_t n = (uint32_t)len;
        if (tid == 0) chain_plan(ctl, a, n);
        T *g = static_cast<T *>(a.data) + o0;
        gather4(copy, tid, blockDim.x, n, [](uint32_t x) { return x; }, [&](uint32_t x) { return g[x]; });
        for (uint32_t x = tid; x < n; x += blockDim.x) ix.head[x] = 0;
        for (uint32_t w = tid; w < (n + 31) / 32; w += blockDim.x) ix.bits[w] = 0;
        __syncthreads();
        if (ctl.nseg == 0) continue;
        const uint32_t lim = chain_limit(n);
        bool ok = true;
        roll_plan_range_src<SRC>(ctl.seg, ctl.nseg, 0, ctl.n_batches, seed, ctl.err,
                                 [&](uint32_t pos, uint32_t v) { ok = chain_push(ix, pos, v, lim) && ok; });
        __syncthreads();
        for (uint32_t y = tid; y < n; y += blockDim.x) ok = chain_fix<false>(ix, y, lim) && ok;
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
struct ChainGridArgs {
    Seg seg[kMaxSegs];
    int nseg;
    uint64_t n_batches;
    uint64_t seed;
    uint32_t *head, *next, *bits;
    void *data, *copy;
    uint32_t n;
    uint32_t *j_out;
    const uint32_t *j_in;  // swap indices given (not rolled): pass 1 pushes them
    uint32_t *bar;  // [2] grid barrier, zero on entry
    int *err;
};

// The phases, each a grid-stride loop over the launch's threads.  They run
// in one cooperative launch separated by grid barriers (lowest latency), or
// as one launch each (no co-residency needed, so they share the GPU with
// kernels on other streams).  If a barrier gives up, or an error is
// recorded, the gather does not run and the array is left as it was.
template <typename T>
__device__ __forceinline__ void grid_phase(const ChainGridArgs &a, int phase, uint64_t gid, uint64_t stride) {
    const GlobalIdx ix{a.head, a.next, a.bits};
    const uint32_t lim = chain_limit(a.n);
    T *A = static_cast<T *>(a.data);
    T *copy = static_cast<T *>(a.copy);
    bool ok = true;
    if (phase == 0) {
        gather4(copy, gid, stride, a.n, [](uint32_t x) { return x; }, [&](uint32_t x) { return A[x]; });
        for (uint64_t x = gid; x < a.n; x += stride) a.head[x] = 0;
        for (uint64_t w = gid; w < ((uint64_t)a.n + 31) / 32; w += stride) a.bits[w] = 0;
    } else if (phase == 1 && a.j_in) {
        for (uint64_t c = gid + 1; c < a.n; c += stride) ok = chain_push(ix, (uint32_t)c, a.j_in[c], lim) && ok;
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
            if (!chain_fix<true>(ix, (uint32_t)y, lim)) ok = false;
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
// Size classes of the CTA kernel: 0 small (128 threads), 1 medium (256),
// 2 large (1024, all of the shared memory).  Their attributes and
// occupancy are set once per context and element size (and again after
// brr_tune moves a class boundary).
constexpr int kClassThreads[3] = {128, 256, 1024};

// The small and medium classes stage every array whole, so they run the
// instance whose accesses are all shared-memory ones.
template <typename T, uint32_t SRC = BRR_WORDS_SPLITMIX64>
static const void *cta_kernel_of(int cls) {
    return cls == 0 ? (const void *)chain_cta_kernel<T, 128, SRC, true>
                    : cls == 1 ? (const void *)chain_cta_kernel<T, 256, SRC, true>
                               : (const void *)chain_cta_kernel<T, 1024, SRC>;
}

template <typename T>
static brr_status chain_setup(brr_ctx *ctx) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    if (ctx->chain_ready[ix]) return BRR_OK;
    const size_t limit = ((size_t)ctx->max_smem_optin - sizeof(ChainCtl) - 1024) & ~(size_t)15;
    uint32_t full = (uint32_t)std::min<size_t>(limit / (sizeof(T) + 4), kChainCtaCap);
    while (full > 0 && CtaLayout(full, sizeof(T)).staged_bytes(full) > limit) full--;
    // heads and bitmap of an unstaged array must fit, with a few links
    uint32_t hi_l = kChainCtaCap;
    while (hi_l > full && CtaLayout(hi_l, 0).next + 16 > limit) hi_l -= 8;
    const uint32_t hi_s = (uint32_t)std::min<uint64_t>(ctx->tune.small_max, full);
    const uint32_t hi_m = std::max(hi_s, (uint32_t)std::min<uint64_t>(ctx->tune.medium_max, full));
    brr_ctx::ChainClass cls[3];
    cls[0] = {0, hi_s, hi_s, 0, CtaLayout(hi_s, sizeof(T)).staged_bytes(hi_s), 0};
    cls[1] = {hi_s, hi_m, hi_m, 0, CtaLayout(hi_m, sizeof(T)).staged_bytes(hi_m), 0};
    cls[2] = {hi_m, std::max(hi_m, hi_l), full, (uint32_t)limit, limit, 0};
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
    ctx->chain_long_per_sm[ix] = long_per_sm;
    ctx->chain_ready[ix] = true;
    return BRR_OK;
}

// One CTA-kernel launch of class c; `single` (one array) takes any length up
// to the class's limit.  Kernels of the other word sources get the class's
// shared-memory attribute on their first launch.
template <typename T, uint32_t SRC>
static cudaError_t launch_cta_class(brr_ctx *ctx, int c, const ChainArgs &a, uint32_t grid,
                                    bool validate, bool single, cudaStream_t stream, uint32_t lo = 0) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    const brr_ctx::ChainClass &k = ctx->chain_cls[ix][c];
    // lo (when given) replaces the class's lower bound: the large class can take
    // any array up to its limit, staged whole up to full_cap
    const CtaClass cls = {single ? 0u : (lo ? lo : k.lo), k.hi, k.full_cap, k.link_bytes, (uint32_t)c,
                          validate ? 1u : 0u};
    if (SRC != BRR_WORDS_SPLITMIX64) {
        const cudaError_t e = cudaFuncSetAttribute(cta_kernel_of<T, SRC>(c),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
        if (e != cudaSuccess) return e;
    }
    if (c == 0) chain_cta_kernel<T, 128, SRC, true><<<grid, 128, k.smem, stream>>>(a, cls);
    else if (c == 1) chain_cta_kernel<T, 256, SRC, true><<<grid, 256, k.smem, stream>>>(a, cls);
    else chain_cta_kernel<T, 1024, SRC><<<grid, 1024, k.smem, stream>>>(a, cls);
    return cudaGetLastError();
}

// Which kernels a staged launch runs, their grids, and the scratch it needs:
// the global slots of the large class (element copies and the links that do
// not fit) and of the long kernel (heads, links, bitmap and copies).
struct StagedPlan {
    bool run[3];
    uint32_t grid[3];
    uint32_t long_grid;
    size_t cta_slot_links, cta_slot_bytes, slot_bytes;
    size_t scratch;
};

template <typename T>
static StagedPlan staged_plan(const brr_ctx *ctx, uint64_t max_len, bool single, uint32_t n_items) {
    const int ix = sizeof(T) == 4 ? 0 : 1;
    const brr_ctx::ChainClass *cls = ctx->chain_cls[ix];
    StagedPlan p = {};
    for (int c = 0; c < 3; c++) {
        p.run[c] = single ? c == 2 : (c == 0 || max_len > cls[c].lo);
        p.grid[c] = (uint32_t)std::min<uint64_t>((uint64_t)cls[c].per_sm * ctx->num_sms, n_items);
    }
    if (p.run[2] && max_len > cls[2].full_cap) {
        const uint64_t most = std::min<uint64_t>(max_len, cls[2].hi);
        p.cta_slot_links = ((size_t)most * sizeof(T) + 255) & ~(size_t)255;
        p.cta_slot_bytes = p.cta_slot_links + (((size_t)most * 2 + 255) & ~(size_t)255);
    }
    if (!single && max_len > kChainCtaCap) {
        p.slot_bytes = SlotLayout(max_len, sizeof(T)).bytes;
        const size_t budget = (size_t)2 << 30;
        p.long_grid = (uint32_t)std::max<size_t>(
            1, std::min<size_t>({(size_t)ctx->chain_long_per_sm[ix] * ctx->num_sms, (size_t)n_items,
                                 budget / p.slot_bytes}));
    }
    p.scratch = 256 + (size_t)p.grid[2] * p.cta_slot_bytes + (size_t)p.long_grid * p.slot_bytes;
    return p;
}

// Batched shuffles (offsets != nullptr): each array goes to the CTA kernel
// of its size class, or, above 65,536 elements, to the long kernel.  One
// array (offsets == nullptr, at most 65,536 elements): the large-class CTA
// kernel with one CTA.
template <typename T, uint32_t SRC = BRR_WORDS_SPLITMIX64>
static brr_status launch_chains_staged(brr_ctx *ctx, ChainArgs a, uint64_t max_len, cudaStream_t stream) {
    brr_status st = chain_setup<T>(ctx);
    if (st != BRR_OK) return st;
    const bool single = a.offsets == nullptr;
    const uint32_t n_items = single ? 1u : a.n_arrays;
    a.max_len = (uint32_t)max_len;
    a.err = ctx->d_err;
    a.ordered_push = (uint32_t)ctx->tune.ordered_push;
    const StagedPlan plan = staged_plan<T>(ctx, max_len, single, n_items);
    a.cta_slot_links = plan.cta_slot_links;
    a.cta_slot_bytes = plan.cta_slot_bytes;
    a.slot_bytes = plan.slot_bytes;
    const size_t cta_slots = (size_t)plan.grid[2] * plan.cta_slot_bytes;
    // batched: the arrays are first sorted into per-class lists, so that a
    // class kernel takes only its own arrays from its counter (no pass over
    // every array per class); under graph capture without room reserved for
    // the lists, the kernels take every array and skip the others'
    // (at most kChainBinMaxArrays arrays: the lists take 28 bytes per array)
    bool binned = !single && a.n_arrays <= kChainBinMaxArrays;
    const size_t bins_bytes = binned ? ((size_t)kChainBinClasses * a.n_arrays * 4 + 255) & ~(size_t)255 : 0;
    const int ix = sizeof(T) == 4 ? 0 : 1;
    const brr_ctx::ChainClass *k = ctx->chain_cls[ix];
    const bool route = !single && ctx->tune.window_route;
    const uint32_t eb = (uint32_t)sizeof(T);
    // windowed reservations (windows.cu) take the small class and every
    // larger array that stages whole: in 256-thread CTAs up to cap_q, in
    // 512-thread CTAs up to cap_mid, in 1024-thread CTAs up to cap, and,
    // with the targets in a global slot per CTA (binned calls that can have
    // the slots), only the elements staged, up to cap_xl; chain resolution
    // the rest
    const uint32_t cap_q = route ? std::max(k[0].hi, windows_quarter_cap(ctx, eb)) : 0u;
    const uint32_t cap_mid = route ? std::max(cap_q, windows_mid_cap(ctx, eb)) : 0u;
    const uint32_t cap = route ? std::max(cap_mid, windows_stage_cap(ctx, eb)) : k[1].hi;
    bool xl = route && binned && max_len > cap;
    const size_t xl_bytes = xl ? (size_t)windows_xl_grid(ctx) * kChainCtaCap * sizeof(uint16_t) : 0;
    st = ensure_scratch(ctx, plan.scratch + bins_bytes + xl_bytes, stream);
    if (st == BRR_EINVAL && xl) {
        xl = false;
        st = ensure_scratch(ctx, plan.scratch + bins_bytes, stream);
    }
    if (st == BRR_EINVAL && binned) {
        binned = false;
        st = ensure_scratch(ctx, plan.scratch, stream);
    }
    if (st != BRR_OK) return st;
    const uint32_t cap_xl = xl ? std::max(cap, windows_xl_cap(ctx, eb)) : cap;
    unsigned char *base = static_cast<unsigned char *>(ctx->scratch);
    a.queue = reinterpret_cast<uint32_t *>(base);  // [0..15] work counters, [16..31] class sizes
    a.cta_slots = base + 256;
    a.slots = base + 256 + cta_slots;
    uint16_t *jt_slots = xl ? reinterpret_cast<uint16_t *>(base + plan.scratch + bins_bytes) : nullptr;
    cudaError_t e = cudaMemsetAsync(a.queue, 0, 32 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    const bool win_small = route && k[0].hi <= kWinSmallMax;  // a small class the windows stage
    if (binned) {
        ChainBins b = {};
        if (route) {
            b.n_cls = 7;
            const uint64_t bd[6] = {k[0].hi, cap_q, cap_mid, cap, cap_xl, kChainCtaCap};
            const uint32_t cl[7] = {win_small ? 4u : 0u, 7, 6, 5, 8, 2, 3};
            for (int i = 0; i < 7; i++) b.cls[i] = cl[i];
            for (int i = 0; i < 6; i++) b.bound[i] = bd[i];
        } else {
            b.n_cls = 4;
            const uint64_t bd[3] = {k[0].hi, k[1].hi, kChainCtaCap};
            const uint32_t cl[4] = {0, 1, 2, 3};
            for (int i = 0; i < 4; i++) b.cls[i] = cl[i];
            for (int i = 0; i < 3; i++) b.bound[i] = bd[i];
        }
        uint32_t *list = reinterpret_cast<uint32_t *>(base + plan.scratch);
        a.bin_list = list;
        a.bin_count = a.queue + 16;
        const uint32_t bgrid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((a.n_arrays + 255) / 256, 4096));
        chain_bin_kernel<<<bgrid, 256, 0, stream>>>(a.offsets, a.n_arrays, max_len, b, list, a.queue + 16, ctx->d_err);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    if (plan.long_grid) {
        chain_long_kernel<T, SRC><<<plan.long_grid, kChainThreads, 0, stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    if (route) {
        // large arrays first: chain large, windows (targets in global memory,
        // large, middle, quarter), small
        auto list_of = [&](uint32_t c) { return binned ? a.bin_list + (size_t)c * a.n_arrays : nullptr; };
        auto count_of = [&](uint32_t c) { return binned ? a.bin_count + c : nullptr; };
        if (max_len > cap_xl) {
            e = launch_cta_class<T, SRC>(ctx, 2, a, plan.grid[2], false, false, stream, cap_xl);
            if (e != cudaSuccess) return cuda_status(e);
        }
        if (xl) {
            st = launch_windows_range(ctx, a.data, a.offsets, a.n_arrays, eb, a.seeds, max_len, a.nk, a.k_max, 4,
                                      cap, cap_xl, a.queue + 8, list_of(8), count_of(8), false, stream, SRC,
                                      jt_slots);
            if (st != BRR_OK) return st;
        }
        st = launch_windows_range(ctx, a.data, a.offsets, a.n_arrays, eb, a.seeds, max_len, a.nk, a.k_max, 2, cap_mid,
                                  cap, a.queue + 5, list_of(5), count_of(5), false, stream, SRC);
        if (st != BRR_OK) return st;
        st = launch_windows_range(ctx, a.data, a.offsets, a.n_arrays, eb, a.seeds, max_len, a.nk, a.k_max, 1, cap_q,
                                  cap_mid, a.queue + 6, list_of(6), count_of(6), false, stream, SRC);
        if (st != BRR_OK) return st;
        st = launch_windows_range(ctx, a.data, a.offsets, a.n_arrays, eb, a.seeds, max_len, a.nk, a.k_max, 3, k[0].hi,
                                  cap_q, a.queue + 7, list_of(7), count_of(7), false, stream, SRC);
        if (st != BRR_OK) return st;
        if (!win_small) {
            e = launch_cta_class<T, SRC>(ctx, 0, a, plan.grid[0], !binned, false, stream);
            return cuda_status(e);
        }
        return launch_windows_range(ctx, a.data, a.offsets, a.n_arrays, eb, a.seeds, max_len, a.nk, a.k_max, 0, 0,
                                    k[0].hi, a.queue + 4, list_of(4), count_of(4), !binned, stream, SRC);
    }
    // large arrays first; without lists the small class validates every array
    for (int c = 2; c >= 0; c--) {
        if (!plan.run[c]) continue;
        e = launch_cta_class<T, SRC>(ctx, c, a, plan.grid[c], (c == 0 && !binned) || single, single, stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return BRR_OK;
}

template <uint32_t SRC>
static brr_status launch_chains_staged_eb(brr_ctx *ctx, const ChainArgs &a, uint32_t elem_bytes, uint64_t max_len,
                                          cudaStream_t stream) {
    return elem_bytes == 4 ? launch_chains_staged<uint32_t, SRC>(ctx, a, max_len, stream)
                           : launch_chains_staged<uint64_t, SRC>(ctx, a, max_len, stream);
}

brr_status launch_chains_batched(brr_ctx *ctx, void *data, const uint64_t *offsets, uint32_t n_arrays,
                                 uint32_t elem_bytes, const uint64_t *seeds, uint64_t max_len,
                                 const brr_schedule *sched, cudaStream_t stream, uint32_t source) {
    ChainArgs a = {};
    a.data = data;
    a.offsets = offsets;
    a.seeds = seeds;
    a.n_arrays = n_arrays;
    for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = sched->n_k[k];
    a.k_max = sched->k_max;
    if (source == BRR_WORDS_CHACHA20)
        return launch_chains_staged_eb<BRR_WORDS_CHACHA20>(ctx, a, elem_bytes, max_len, stream);
    if (source == BRR_WORDS_SPLITMIX32)
        return launch_chains_staged_eb<BRR_WORDS_SPLITMIX32>(ctx, a, elem_bytes, max_len, stream);
    return launch_chains_staged_eb<BRR_WORDS_SPLITMIX64>(ctx, a, elem_bytes, max_len, stream);
}

// Grid-path scratch: barrier words, heads, links, bitmap, copy of the array.
struct GridLayout {
    size_t head, next, bits, copy, bytes;
    GridLayout(uint64_t n, uint32_t eb) {
        const size_t links = ((size_t)n * 4 + 255) & ~(size_t)255;
        head = 256;
        next = head + links;
        bits = next + links;
        copy = bits + ((((size_t)n + 31) / 32 * 4 + 255) & ~(size_t)255);
        bytes = copy + (((size_t)n * eb + 255) & ~(size_t)255);
    }
};

size_t chains_grid_scratch(uint64_t n, uint32_t elem_bytes) { return GridLayout(n, elem_bytes).bytes; }

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
// bytes), in one cooperative launch or in five launches.  With j_in the swap
// indices are read from it instead of rolled.
brr_status launch_chains_grid(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                              const brr_schedule *sched, uint32_t *j_out, void *scratch, int *err,
                              int num_sms, cudaStream_t stream, bool cooperative, const uint32_t *j_in) {
    ChainGridArgs a;
    a.j_in = j_in;
    a.nseg = plan_segments(n, 1, sched->n_k, sched->k_max, a.seg, kMaxSegs, &a.n_batches);
    if (a.nseg < 0) return BRR_EINVAL;
    a.seed = seed;
    a.n = (uint32_t)n;
    a.j_out = j_out;
    a.err = err;
    a.data = data;
    const GridLayout lay(n, elem_bytes);
    unsigned char *base = static_cast<unsigned char *>(scratch);
    a.bar = reinterpret_cast<uint32_t *>(base);
    a.head = reinterpret_cast<uint32_t *>(base + lay.head);
    a.next = reinterpret_cast<uint32_t *>(base + lay.next);
    a.bits = reinterpret_cast<uint32_t *>(base + lay.bits);
    a.copy = base + lay.copy;
    const int per_sm = chain_grid_per_sm(elem_bytes);
    if (per_sm < 1) return BRR_ECUDA;
    cudaError_t e;
    if (!cooperative) {
        const uint64_t cap = (uint64_t)per_sm * num_sms;
        for (int phase = 0; phase < 5; phase++) {
            const uint64_t units = phase == 1 && !j_in ? a.n_batches : n;
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
    // enough blocks for one position (or batch) per thread, at most all resident
    const uint64_t want = (std::max<uint64_t>(n, a.n_batches) + kChainGridThreads - 1) / kChainGridThreads;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)per_sm * num_sms));
    e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    void *args[] = {&a};
    e = elem_bytes == 4
        ? cudaLaunchCooperativeKernel((const void *)chain_grid_kernel<uint32_t>, grid, kChainGridThreads, args, 0, stream)
        : cudaLaunchCooperativeKernel((const void *)chain_grid_kernel<uint64_t>, grid, kChainGridThreads, args, 0, stream);
    return cuda_status(e);
}

// One array: one CTA up to tune.single_cta_max elements (at most 65,536),
// else the grid passes.
brr_status launch_chains_one(brr_ctx *ctx, void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                             const brr_schedule *sched, uint32_t *j_out, cudaStream_t stream) {
    const int ix = elem_bytes == 4 ? 0 : 1;
    brr_status st = elem_bytes == 4 ? chain_setup<uint32_t>(ctx) : chain_setup<uint64_t>(ctx);
    if (st != BRR_OK) return st;
    if (n <= std::min<uint64_t>(ctx->tune.single_cta_max, ctx->chain_cls[ix][2].hi)) {
        ChainArgs a = {};
        a.data = data;
        a.n_arrays = 1;
        a.single_n = (uint32_t)n;
        a.single_seed = seed;
        a.j_out = j_out;
        for (int k = 0; k <= BRR_SCHED_KMAX; k++) a.nk[k] = sched->n_k[k];
        a.k_max = sched->k_max;
        return elem_bytes == 4 ? launch_chains_staged<uint32_t>(ctx, a, n, stream)
                               : launch_chains_staged<uint64_t>(ctx, a, n, stream);
    }
    st = ensure_scratch(ctx, chains_grid_scratch(n, elem_bytes), stream);
    if (st != BRR_OK) return st;
    return launch_chains_grid(data, n, elem_bytes, seed, sched, j_out, ctx->scratch, ctx->d_err,
                              ctx->num_sms, stream, ctx->tune.grid_cooperative != 0);
}

// Scratch for every chain-resolution shuffle of up to max_len elements (one
// array or any number of batched arrays, 4- or 8-byte elements); also sets
// up the kernels' attributes, so that later calls need no setup.
brr_status chains_reserve(brr_ctx *ctx, uint64_t max_len, size_t *bytes) {
    size_t most = 0;
    for (uint32_t eb : {4u, 8u}) {
        const brr_status st = eb == 4 ? chain_setup<uint32_t>(ctx) : chain_setup<uint64_t>(ctx);
        if (st != BRR_OK) return st;
        if (max_len == 0) continue;
        const StagedPlan a = eb == 4 ? staged_plan<uint32_t>(ctx, max_len, false, 0xFFFFFFFFu)
                                     : staged_plan<uint64_t>(ctx, max_len, false, 0xFFFFFFFFu);
        const StagedPlan b = eb == 4 ? staged_plan<uint32_t>(ctx, max_len, true, 1)
                                     : staged_plan<uint64_t>(ctx, max_len, true, 1);
        most = std::max({most, a.scratch, b.scratch, chains_grid_scratch(max_len, eb)});
    }
    *bytes = most;
    return BRR_OK;
}

}  // namespace brr
