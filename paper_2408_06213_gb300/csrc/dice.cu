// dice.cu -- bulk batched dice (Section 5): Algorithm 3 (per-roll bounds,
// threshold computed on the rare path) and Algorithm 2 (one fixed bound,
// threshold known in advance), as persistent kernels over tiles of batches.
//
// Per tile a CTA stages the batch offsets and bounds in shared memory, runs
// one Theorem 1 chain per batch (one thread per batch), writes the digits to
// a shared-memory copy of the tile's output, compacts the rejected batches
// with a warp ballot into a CTA-local list and reruns only those with the
// next attempt word until the list is empty, then stores the tile with
// coalesced writes.  Rejections never touch global memory and never
// serialise the word stream: attempt a of batch g is always word(seed, g, a).
#include <algorithm>

#include "brr_common.cuh"
#include "internal.h"

namespace brr {

constexpr int kDiceThreads = 256;
constexpr int kVarTileBatches = 1024;  // batches per tile, per-roll bounds
constexpr int kTileRollsCap = 8192;    // rolls staged per tile

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

struct DiceSmem {
    uint32_t off[kVarTileBatches + 1];
    uint32_t bm1[kTileRollsCap];
    uint32_t out[kTileRollsCap];
    uint16_t list[2][kTileRollsCap];
    int cnt[2];
    int err;
};

// Warp-aggregated append of `flag` lanes' values to a shared-memory list.
__device__ __forceinline__ void warp_append(bool flag, uint16_t value, uint16_t *list, int *cnt) {
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) list[base + __popc(mask & ((1u << lane) - 1))] = value;
}

// One Algorithm 3 attempt for a batch whose bounds (as b - 1) are staged in
// shared memory at [s, e): writes the digits, returns whether the attempt is
// accepted.  *valid is cleared if the batch product exceeds 2^64.
__device__ __forceinline__ bool var_attempt(const uint32_t *sbm1, uint32_t *sout, uint32_t s,
                                            uint32_t e, uint64_t seed, uint64_t g, uint32_t att,
                                            bool *valid) {
    uint64_t r = word(seed, g, att);
    uint64_t Bm1 = 0;
    bool ok = true;
    for (uint32_t x = s; x < e; x++) {
        const uint32_t m1 = sbm1[x];
        sout[x] = chain_step_m1(r, m1);
        ok = prod_m1_step(Bm1, m1) && ok;
    }
    *valid = ok;
    // r >= B accepts at once (the threshold is below B); otherwise compare
    // with the exact threshold 2^64 mod B.
    return r > Bm1 || r >= threshold_from_m1(Bm1);
}

// Same, reading bounds from and writing digits to global memory (used only
// for tiles whose rolls do not fit the staging buffer).
__device__ bool var_attempt_global(const uint32_t *bm1, uint32_t *out, uint64_t s, uint64_t e,
                                   uint64_t seed, uint64_t g, uint32_t att, bool *valid) {
    uint64_t r = word(seed, g, att);
    uint64_t Bm1 = 0;
    bool ok = true;
    for (uint64_t x = s; x < e; x++) {
        const uint32_t m1 = bm1[x];
        out[x] = chain_step_m1(r, m1);
        ok = prod_m1_step(Bm1, m1) && ok;
    }
    *valid = ok;
    return r > Bm1 || r >= threshold_from_m1(Bm1);
}

// Per-roll bounds.  kImplicit: batch g is roll g (unbatched form, off unused).
template <bool kImplicit>
__global__ void __launch_bounds__(kDiceThreads)
dice_var_kernel(const uint32_t *__restrict__ bm1, const uint32_t *__restrict__ off,
                uint64_t n_batches, uint64_t n_rolls, uint64_t seed, uint32_t *__restrict__ out,
                int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DiceSmem &S = *reinterpret_cast<DiceSmem *>(smem_raw);
    const int tid = threadIdx.x;
    constexpr uint32_t TB = kImplicit ? (uint32_t)kTileRollsCap : (uint32_t)kVarTileBatches;
    const uint64_t n_tiles = (n_batches + TB - 1) / TB;
    if (tid == 0) S.err = 0;

    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t g0 = tile * TB;
        const uint32_t nb = (uint32_t)umin64(TB, n_batches - g0);
        // ---- stage offsets
        if (!kImplicit) {
            for (uint32_t x = tid; x <= nb; x += kDiceThreads) S.off[x] = off[g0 + x];
        }
        if (tid == 0) { S.cnt[0] = 0; S.cnt[1] = 0; }
        __syncthreads();
        uint64_t r0, r1;
        bool tile_ok = true;
        if (kImplicit) {
            r0 = g0;
            r1 = g0 + nb;
        } else {
            r0 = S.off[0];
            r1 = S.off[nb];
            if (r1 < r0 || r1 > n_rolls) tile_ok = false;
            if (tile == 0 && r0 != 0) tile_ok = false;
            if (g0 + nb == n_batches && r1 != n_rolls) tile_ok = false;
        }
        if (!tile_ok) {
            if (tid == 0) S.err = BRR_EINVAL;
            __syncthreads();
            continue;
        }
        const uint32_t nr = (uint32_t)(r1 - r0);
        if (nr <= (uint32_t)kTileRollsCap) {
            // ---- stage bounds (coalesced)
            for (uint32_t x = tid; x < nr; x += kDiceThreads) S.bm1[x] = bm1[r0 + x];
            __syncthreads();
            // ---- first pass: one batch per thread, uniform trip count
            bool bad = false;
            for (uint32_t base = 0; base < nb; base += kDiceThreads) {
                const uint32_t b = base + tid;
                bool rej = false;
                if (b < nb) {
                    uint32_t s, e;
                    if (kImplicit) { s = b; e = b + 1; }
                    else {
                        s = S.off[b] - (uint32_t)r0;
                        e = S.off[b + 1] - (uint32_t)r0;
                        if (e < s || e > nr) { bad = true; e = s; }
                    }
                    bool valid;
                    const bool acc = var_attempt(S.bm1, S.out, s, e, seed, g0 + b, 0, &valid);
                    bad |= !valid;
                    rej = !acc;
                }
                warp_append(rej, (uint16_t)b, S.list[0], &S.cnt[0]);
            }
            if (bad) S.err = BRR_EINVAL;
            // ---- retry passes over the compacted rejected batches
            int cur = 0;
            uint32_t att = 1;
            __syncthreads();
            while (S.cnt[cur] != 0) {
                if (att >= kMaxAttempts) {
                    if (tid == 0) S.err = BRR_ERETRY;
                    break;
                }
                const int cnt = S.cnt[cur];
                __syncthreads();
                if (tid == 0) S.cnt[cur ^ 1] = 0;
                __syncthreads();
                for (int base = 0; base < cnt; base += kDiceThreads) {
                    const int idx = base + tid;
                    bool rej = false;
                    uint32_t b = 0;
                    if (idx < cnt) {
                        b = S.list[cur][idx];
                        uint32_t s, e;
                        if (kImplicit) { s = b; e = b + 1; }
                        else {
                            s = S.off[b] - (uint32_t)r0;
                            e = S.off[b + 1] - (uint32_t)r0;
                            if (e < s || e > nr) e = s;
                        }
                        bool valid;
                        rej = !var_attempt(S.bm1, S.out, s, e, seed, g0 + b, att, &valid);
                    }
                    warp_append(rej, (uint16_t)b, S.list[cur ^ 1], &S.cnt[cur ^ 1]);
                }
                __syncthreads();
                cur ^= 1;
                att++;
            }
            __syncthreads();
            // ---- coalesced store of the tile
            for (uint32_t x = tid; x < nr; x += kDiceThreads) out[r0 + x] = S.out[x];
        } else {
            // Tile too long to stage (many dice of bound 1): one thread per
            // batch straight from global memory, retrying in place.
            for (uint32_t b = tid; b < nb; b += kDiceThreads) {
                const uint64_t s = S.off[b], e = S.off[b + 1];
                if (e < s || e > n_rolls) { S.err = BRR_EINVAL; continue; }
                uint32_t att = 0;
                bool valid = true, acc = false;
                while (!acc && att < kMaxAttempts) {
                    acc = var_attempt_global(bm1, out, s, e, seed, g0 + b, att, &valid);
                    if (!valid) break;
                    att++;
                }
                if (!valid) S.err = BRR_EINVAL;
                else if (!acc) S.err = BRR_ERETRY;
            }
        }
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0 && S.err) record_error(err, S.err);
}

// One fixed bound b = bm1 + 1 in batches of k (Algorithm 2).  Tiles hold
// `tb` batches (a multiple of 4, tb * k <= kTileRollsCap); the last batch of
// the stream may be short and uses t_last.
__global__ void __launch_bounds__(kDiceThreads)
dice_fixed_kernel(uint32_t bm1, uint32_t k, uint32_t tb, uint64_t t_full, uint64_t t_last,
                  uint64_t n_rolls, uint64_t seed, uint32_t *__restrict__ out, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DiceSmem &S = *reinterpret_cast<DiceSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const uint64_t n_batches = (n_rolls + k - 1) / k;
    const uint64_t n_tiles = (n_batches + tb - 1) / tb;
    if (tid == 0) S.err = 0;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t g0 = tile * tb;
        const uint32_t nb = (uint32_t)umin64(tb, n_batches - g0);
        const uint64_t r0 = g0 * k;
        const uint32_t nr = (uint32_t)(umin64(n_rolls, (g0 + nb) * k) - r0);
        if (tid == 0) { S.cnt[0] = 0; S.cnt[1] = 0; }
        __syncthreads();
        for (uint32_t base = 0; base < nb; base += kDiceThreads) {
            const uint32_t b = base + tid;
            bool rej = false;
            if (b < nb) {
                const uint32_t s = b * k;
                const uint32_t kk = min(k, nr - s);
                const uint64_t t = (kk == k) ? t_full : t_last;
                uint64_t r = word(seed, g0 + b, 0);
                for (uint32_t i = 0; i < kk; i++) S.out[s + i] = chain_step_m1(r, bm1);
                rej = r < t;
            }
            warp_append(rej, (uint16_t)b, S.list[0], &S.cnt[0]);
        }
        int cur = 0;
        uint32_t att = 1;
        __syncthreads();
        while (S.cnt[cur] != 0) {
            if (att >= kMaxAttempts) {
                if (tid == 0) S.err = BRR_ERETRY;
                break;
            }
            const int cnt = S.cnt[cur];
            __syncthreads();
            if (tid == 0) S.cnt[cur ^ 1] = 0;
            __syncthreads();
            for (int base = 0; base < cnt; base += kDiceThreads) {
                const int idx = base + tid;
                bool rej = false;
                uint32_t b = 0;
                if (idx < cnt) {
                    b = S.list[cur][idx];
                    const uint32_t s = b * k;
                    const uint32_t kk = min(k, nr - s);
                    const uint64_t t = (kk == k) ? t_full : t_last;
                    uint64_t r = word(seed, g0 + b, att);
                    for (uint32_t i = 0; i < kk; i++) S.out[s + i] = chain_step_m1(r, bm1);
                    rej = r < t;
                }
                warp_append(rej, (uint16_t)b, S.list[cur ^ 1], &S.cnt[cur ^ 1]);
            }
            __syncthreads();
            cur ^= 1;
            att++;
        }
        __syncthreads();
        for (uint32_t x = tid; x < nr; x += kDiceThreads) out[r0 + x] = S.out[x];
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0 && S.err) record_error(err, S.err);
}

static int persistent_grid(brr_ctx *ctx, const void *kernel, size_t smem, uint64_t n_tiles) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kDiceThreads, smem);
    if (per_sm < 1) per_sm = 1;
    const uint64_t full = (uint64_t)per_sm * (uint64_t)ctx->num_sms;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(full, n_tiles));
}

brr_status launch_dice_var(brr_ctx *ctx, const uint32_t *bm1, const uint32_t *off,
                           uint64_t n_batches, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                           cudaStream_t stream) {
    if (n_batches == 0) return BRR_OK;
    const size_t smem = sizeof(DiceSmem);
    if (off == nullptr) {
        const void *kern = (const void *)dice_var_kernel<true>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const uint64_t n_tiles = (n_batches + kTileRollsCap - 1) / kTileRollsCap;
        const int grid = persistent_grid(ctx, kern, smem, n_tiles);
        dice_var_kernel<true><<<grid, kDiceThreads, smem, stream>>>(bm1, off, n_batches, n_rolls,
                                                                    seed, out, ctx->d_err);
    } else {
        const void *kern = (const void *)dice_var_kernel<false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const uint64_t n_tiles = (n_batches + kVarTileBatches - 1) / kVarTileBatches;
        const int grid = persistent_grid(ctx, kern, smem, n_tiles);
        dice_var_kernel<false><<<grid, kDiceThreads, smem, stream>>>(bm1, off, n_batches, n_rolls,
                                                                     seed, out, ctx->d_err);
    }
    return cuda_status(cudaGetLastError());
}

brr_status launch_dice_fixed(brr_ctx *ctx, uint32_t bm1, uint32_t k, uint64_t t_full,
                             uint64_t t_last, uint64_t n_rolls, uint64_t seed, uint32_t *out,
                             cudaStream_t stream) {
    if (n_rolls == 0) return BRR_OK;
    const size_t smem = sizeof(DiceSmem);
    const void *kern = (const void *)dice_fixed_kernel;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    uint32_t tb = (uint32_t)kTileRollsCap / k;
    tb &= ~3u;                      // keep tile starts 16-byte aligned
    if (tb == 0) tb = 1;
    const uint64_t n_batches = (n_rolls + k - 1) / k;
    const uint64_t n_tiles = (n_batches + tb - 1) / tb;
    const int grid = persistent_grid(ctx, kern, smem, n_tiles);
    dice_fixed_kernel<<<grid, kDiceThreads, smem, stream>>>(bm1, k, tb, t_full, t_last, n_rolls,
                                                            seed, out, ctx->d_err);
    return cuda_status(cudaGetLastError());
}

}  // namespace brr
