/*
 * inputs_group.c -- helper of the seeded input generators (inputs.py).
 *
 * Groups a sequence of per-roll bounds into batches for the bulk-dice
 * workload: scanning left to right, a batch is extended by the next bound
 * while it holds fewer than k_max bounds and the product of its bounds stays
 * at most 2^64 (the condition Theorem 1 places on a batch).  Writes the CSR
 * offsets (n_batches + 1 entries, first 0, last n) and returns n_batches.
 * This is input preparation only; it rolls nothing.
 */
#include <stdint.h>

typedef unsigned __int128 u128;

uint64_t brr_inputs_group(const uint32_t *bm1, uint64_t n, uint32_t k_max, uint32_t *off)
{
    const u128 W = (u128)1 << 64;
    uint64_t nb = 0, x = 0;
    off[0] = 0;
    while (x < n) {
        u128 p = (u128)bm1[x] + 1;
        uint64_t e = x + 1;
        while (e < n && e - x < k_max) {
            u128 q = p * ((u128)bm1[e] + 1);
            if (q > W) break;
            p = q;
            e++;
        }
        off[++nb] = (uint32_t)e;
        x = e;
    }
    return nb;
}
