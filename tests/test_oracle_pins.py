"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values the
paper prints (Table 1, Table 2, the Section 7 schedule), the closed form in
the proof of Theorem 1, exhaustive enumeration at a toy word size, the
textbook single-roll method (Lemma 1), a published SplitMix64 test vector and
statistical equiprobability.  A dropped term, a wrong sign, an index or digit
order mistake, or a wrong threshold anywhere in the oracle fails one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

M64 = (1 << 64) - 1
GOLDEN_RATIO = 0x9E3779B97F4A7C15


# ------------------------------------------------------------ word source --
def test_splitmix64_published_vector(golden):
    # word(seed, 0, t + 1) is output t of sequential SplitMix64 seeded with seed.
    for t, val in golden("splitmix64_seed1234567.txt"):
        assert oracle.word(1234567, 0, t + 1) == val


def test_word_counter_layout():
    # the counter is (g << 16) | a: batch g, attempt a share one finalizer input
    seed = 0xDEADBEEF
    for g, a in [(0, 0), (1, 0), (0, 65535), (12345, 17), ((1 << 48) - 1, 3)]:
        c = ((g << 16) | a) & M64
        assert oracle.word(seed, g, a) == oracle.mix64((seed + GOLDEN_RATIO * c) & M64)
    assert oracle.word(seed, 1, 0) != oracle.word(seed, 0, 1)


# ------------------------------------------------- Theorem 1, worked example --
def test_table1_worked_example(golden):
    rows = golden("table1_worked_example_L4_b2_6.txt")
    assert len(rows) == 16
    assert oracle.threshold(4, [2, 6]) == 4  # 16 mod 12
    for r0, two_r0, a1, r1, six_r1, a2, r2, reject in rows:
        assert two_r0 == 2 * r0 and six_r1 == 6 * r1
        (d1,), s1 = oracle.chain(4, [2], r0)
        assert (d1, s1) == (a1, r1)
        (d, e), s2 = oracle.chain(4, [2, 6], r0)
        assert (d, e, s2) == (a1, a2, r2)
        assert (s2 < oracle.threshold(4, [2, 6])) == bool(reject)
    # 12 accepted rows, one per outcome pair (a1, a2)
    acc = {(r[2], r[5]) for r in rows if not r[7]}
    assert acc == set(itertools.product(range(2), range(6)))


# -------------------------------------------- exhaustive enumeration, L=16 --
def _l16_tuples():
    rng = np.random.default_rng(2408)
    tuples = [(2, 6), (65536,), (256, 256), (3, 5, 7, 11), (2, 3, 4, 5, 6), (16, 16, 16, 16),
              (65535,), (1, 7, 1), (181, 181), (40, 41, 39), (10, 9, 8, 7, 6), (3,) * 10]
    while len(tuples) < 24:
        k = int(rng.integers(1, 6))
        b = [int(x) for x in rng.integers(1, 60, size=k)]
        if math.prod(b) <= 1 << 16:
            tuples.append(tuple(b))
    return tuples


@pytest.mark.parametrize("b", _l16_tuples())
def test_exhaustive_L16_uniform_outcomes(b):
    """Every accepted 16-bit word maps to an outcome tuple, each tuple exactly
    floor(2^16/B) times; exactly 2^16 mod B words are rejected (Theorem 1)."""
    L, W, B = 16, 1 << 16, math.prod(b)
    t = oracle.threshold(L, b)
    assert t == W % B
    counts = {}
    rejected = 0
    for r0 in range(W):
        a, rk = oracle.chain(L, b, r0)
        assert all(0 <= ai < bi for ai, bi in zip(a, b))
        if rk < t:
            rejected += 1
        else:
            counts[tuple(a)] = counts.get(tuple(a), 0) + 1
    assert rejected == W % B
    assert len(counts) == B
    assert set(counts.values()) == {W // B}


# ----------------------------------------------- closed form at L = 64 --
def _mixed_radix_digits(x, b):
    """MSB-first digits of x < prod(b) in base (b_1..b_k), by division."""
    digits = []
    for bi in reversed(b):
        digits.append(x % bi)
        x //= bi
    assert x == 0
    return digits[::-1]


def test_closed_form_L64():
    """Proof of Theorem 1: prod(b) (*) r0 = (a, r_k), a the mixed-radix value
    of the digits, for every word whether accepted or not."""
    rng = np.random.default_rng(7)
    for trial in range(3000):
        k = int(rng.integers(1, 9))
        b = []
        budget = 64
        for _ in range(k):
            e = int(rng.integers(1, min(budget, 33) + 1)) if budget > 0 else 0
            if e == 0:
                break
            b.append(int(rng.integers(1, (1 << e) + 1)) if e < 64 else 1 << 32)
            budget -= max(1, (b[-1] - 1).bit_length())
        if not b or math.prod(b) > 1 << 64:
            continue
        r0 = int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2))
        a, rk = oracle.chain(64, b, r0)
        B = math.prod(b)
        hi, lo = (B * r0) >> 64, (B * r0) & M64
        assert rk == lo
        assert a == _mixed_radix_digits(hi, b)


def test_threshold_definition():
    for b in ([6], [52] * 6, [1000] * 6, [(1 << 31) + 1] * 2, [1 << 32, 1 << 32], [3, 5, 7]):
        B = math.prod(b)
        assert oracle.threshold(64, b) == (1 << 64) % B
    with pytest.raises(oracle.OracleError):
        oracle.threshold(64, [1 << 32, (1 << 32) - 1, 3])


# ------------------------------------------------- k = 1 is Lemma 1 ------
def _lemire_textbook(b, words):
    """Lemire's nearly-divisionless method written from Section 2 with Python
    integers: accept the high half when the low half is >= 2^64 mod b."""
    for r in words:
        x, y = (b * r) >> 64, (b * r) & M64
        if y >= (1 << 64) % b:
            return x
    raise AssertionError("ran out of words")


def test_k1_reduces_to_lemire():
    rng = np.random.default_rng(11)
    bounds = [1, 2, 3, 6, 52, 1000, (1 << 31) + 1, (1 << 32) - 1, 1 << 32] + [
        int(x) for x in rng.integers(1, 1 << 32, size=40)
    ]
    for b in bounds:
        for g in range(25):
            seed = int(rng.integers(0, 1 << 63))
            words = [oracle.word(seed, g, a) for a in range(64)]
            ref = _lemire_textbook(b, words)
            assert oracle.lemire(b, seed, g) == ref
            assert oracle.roll_batch([b], seed, g)[0] == [ref]


def test_unbatched_dice_is_lemire_per_roll():
    rng = np.random.default_rng(12)
    bm1 = rng.integers(0, 1 << 32, size=300, dtype=np.uint64).astype(np.uint32)
    out = oracle.dice(bm1, None, seed=99)
    for x in range(300):
        assert out[x] == oracle.lemire(int(bm1[x]) + 1, 99, x)


def test_known_threshold_equals_unknown_threshold():
    """Algorithm 2 (fixed b, threshold precomputed) and Algorithm 3 (product and
    threshold computed on the rare path) accept the same words."""
    for b, k, n in [(6, 6, 1000), (52, 6, 997), (1000, 6, 500), ((1 << 31) + 1, 2, 801), (1 << 32, 2, 77)]:
        fixed = oracle.dice_fixed(b, k, n, seed=5)
        off = np.minimum(np.arange(0, n + k, k), n).astype(np.uint32)
        off = np.unique(off)
        var = oracle.dice(np.full(n, b - 1, dtype=np.uint32), off, seed=5)
        assert np.array_equal(fixed, var)


def test_product_2_pow_64_always_accepts():
    # b = (2^32, 2^32): threshold 0, the digits are the two halves of the word
    for g in range(50):
        a, att = oracle.roll_batch([1 << 32, 1 << 32], 3, g)
        w = oracle.word(3, g, 0)
        assert att == 1 and a == [w >> 32, w & 0xFFFFFFFF]


def test_invalid_batch_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.dice(np.full(3, 0xFFFFFFFF, dtype=np.uint32), np.array([0, 3], dtype=np.uint32), 1)
    with pytest.raises(oracle.OracleError):
        oracle.dice_fixed(7, 23, 100, 1)  # 7^23 > 2^64


# ----------------------------------------------------- dice statistics --
def _chi2_ok(counts, expected, dof):
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    # loose bound: mean dof, sd sqrt(2 dof); 6 sd is far outside chance
    return chi2 < dof + 6 * math.sqrt(2 * dof), chi2


@pytest.mark.parametrize("b,k", [(6, 6), (52, 6), (1000, 6), ((1 << 31) + 1, 2)])
def test_dice_fixed_chi_square(b, k):
    n = 60000
    out = oracle.dice_fixed(b, k, n, seed=7).astype(np.uint64)
    assert out.max() < b
    bins = min(b, 64)
    # fold into equal-mass bins (exact when bins divides b; otherwise by value range)
    if b % bins == 0:
        idx = out % bins
    else:
        idx = (out * bins) // b
        # bin sizes differ by at most one value
    counts = np.bincount(idx.astype(np.int64), minlength=bins).astype(float)
    sizes = np.array([((v + 1) * b + bins - 1) // bins - (v * b + bins - 1) // bins for v in range(bins)], float)
    if b % bins == 0:
        sizes = np.full(bins, b // bins, float)
    ok, chi2 = _chi2_ok(counts, n * sizes / b, bins - 1)
    assert ok, chi2


# ------------------------------------------------------------ shuffles --
def test_schedule_is_table2_rounded_down(golden):
    table = {(L, k): v for L, k, v in golden("table2_estimated_nk.txt")}
    for k, nk in golden("experiment_schedule.txt"):
        assert oracle.PAPER_NK[k] == nk
        assert nk <= table[(64, k)] < 2 * nk  # next-lower power of two


def test_k_rule_matches_section7_text():
    # batches of 2 when n <= 2^30, 3 when n <= 2^19, 4 when <= 2^14, 5 <= 2^11, 6 <= 2^9
    for i, k in [((1 << 30) + 1, 1), (1 << 30, 2), ((1 << 19) + 1, 2), (1 << 19, 3), ((1 << 14) + 1, 3),
                 (1 << 14, 4), ((1 << 11) + 1, 4), (1 << 11, 5), (513, 5), (512, 6), (7, 6), (2, 6)]:
        assert oracle.k_rule(i) == k
    assert oracle.k_rule(100, k_max=1) == 1
    assert oracle.k_rule(100, k_max=2) == 2


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_shuffle_exhaustive_L16(n):
    """Algorithm 1 with one Algorithm 4 batch (dice n..2) at L = 16: every one of
    the n! permutations is produced by exactly floor(2^16/n!) words, whatever
    valid upper bound u the fast path uses (Section 6)."""
    W, B = 1 << 16, math.factorial(n)
    for u in (B, 2 * B + 1, W - 1):
        counts = {}
        rejected = 0
        for r0 in range(W):
            z = np.arange(n, dtype=np.uint64)
            acc, _ = oracle.partial_shuffle_word_L(16, z, n, n - 1, u, r0)
            if acc:
                counts[tuple(int(x) for x in z)] = counts.get(tuple(int(x) for x in z), 0) + 1
            else:
                rejected += 1
        assert rejected == W % B
        assert len(counts) == B
        assert set(counts.values()) == {W // B}


def test_shuffle_L64_equiprobable_small_n():
    # n = 4: 24 permutations over 24000 seeds, chi-square
    counts = {}
    for seed in range(24000):
        z, _ = oracle.shuffle(np.arange(4, dtype=np.uint32), seed)
        counts[tuple(z)] = counts.get(tuple(z), 0) + 1
    assert len(counts) == 24
    ok, chi2 = _chi2_ok(np.array(list(counts.values()), float), np.full(24, 1000.0), 23)
    assert ok, chi2


def test_shuffle_position_value_chi_square():
    n, trials = 50, 4000
    counts = np.zeros((n, n))
    base = np.arange(n, dtype=np.uint32)
    for s in range(trials):
        z, _ = oracle.shuffle(base, 1000 + s)
        counts[np.arange(n), z] += 1
    ok, chi2 = _chi2_ok(counts.ravel(), np.full(n * n, trials / n), n * n - 1)
    assert ok, chi2


@pytest.mark.parametrize("n", [0, 1, 2, 3, 7, 100, 513, 2049, 20000])
def test_shuffle_permutation_and_j(n):
    data = np.arange(n, dtype=np.uint64) * 3 + 1
    z, j = oracle.shuffle(data, 42)
    assert np.array_equal(np.sort(z), data)
    assert np.all(j <= np.arange(n))
    assert np.array_equal(oracle.apply_swaps(data, j), z)


def test_unbatched_shuffle_is_textbook_fisher_yates():
    # k_max = 1: j[p] is Lemire's roll of bound p+1 on the words of batch n-1-p
    n, seed = 300, 17
    _, j = oracle.shuffle(np.arange(n, dtype=np.uint32), seed, k_max=1)
    for p in range(n - 1, 0, -1):
        assert j[p] == oracle.lemire(p + 1, seed, n - 1 - p)


def test_batched_shuffle_digits_follow_algorithm4():
    # first batch of a shuffle of n = 1000 (k = 5): dice 1000, 999, ..., 996
    n, seed = 1000, 9
    _, j = oracle.shuffle(np.arange(n, dtype=np.uint32), seed)
    a, _ = oracle.roll_batch([1000, 999, 998, 997, 996], seed, 0)
    assert [int(j[n - 1 - m]) for m in range(5)] == a


def test_shuffle_batched_matches_loop():
    rng = np.random.default_rng(3)
    sizes = rng.integers(0, 300, size=20)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    data = rng.integers(0, 1 << 32, size=int(offsets[-1]), dtype=np.uint64).astype(np.uint32)
    seeds = rng.integers(0, 1 << 63, size=20, dtype=np.uint64)
    out = oracle.shuffle_batched(data, offsets, seeds)
    for s in range(20):
        a, b = int(offsets[s]), int(offsets[s + 1])
        z, _ = oracle.shuffle(data[a:b], int(seeds[s]))
        assert np.array_equal(out[a:b], z)


# --------------------------------------------------------------- samples --
@pytest.mark.parametrize("n", [1, 2, 5, 9, 600, 3000])
def test_sample_full_equals_shuffle(n):
    z, _ = oracle.shuffle(np.arange(n, dtype=np.uint32), 77)
    for m in (n, n - 1):
        if m < 0:
            continue
        s = oracle.sample(n, m, 77)
        assert np.array_equal(s, z[::-1][:m])


def test_sample_prefix_property():
    # sample(n, m) shares all but its last (truncated) batch with sample(n, m')
    n, seed = 5000, 123
    big = oracle.sample(n, 400, seed)
    for m in (1, 2, 5, 6, 7, 30, 399):
        s = oracle.sample(n, m, seed)
        assert len(set(s.tolist())) == m and s.max() < n
        # the first batches have size 5 here (n <= 2^11), so all but the last
        # partial batch agree
        full = (m // 5) * 5 if m % 5 else m
        assert np.array_equal(s[:full], big[:full])


def test_sample_first_draw_uniform():
    n, trials = 20, 20000
    counts = np.bincount([int(oracle.sample(n, 3, s)[0]) for s in range(trials)], minlength=n)
    ok, chi2 = _chi2_ok(counts.astype(float), np.full(n, trials / n), n - 1)
    assert ok, chi2


def test_sample_edge_cases():
    assert oracle.sample(10, 0, 1).size == 0
    assert oracle.sample(1, 1, 1).tolist() == [0]
    with pytest.raises(oracle.OracleError):
        oracle.sample(5, 6, 1)


# ------------------------------------------------------------ cost model --
def test_table2_fast_columns(golden):
    for L, k, v in golden("table2_estimated_nk.txt"):
        if (L, k) == (64, 2):
            continue  # covered by the slow test below
        assert oracle.nk(k, L) == v


@pytest.mark.slow
def test_table2_L64_k2(golden):
    (v,) = [v for L, k, v in golden("table2_estimated_nk.txt") if (L, k) == (64, 2)]
    assert oracle.nk(2, 64) == v
