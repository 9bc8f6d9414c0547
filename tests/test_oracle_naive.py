"""Pins of the oracle's naive batched shuffle (the paper's division-based
comparison method, Section 3 and its appendix listing): one Lemire roll of
the product of a batch's dice, split into the dice by remainders of
successive quotients, least significant first."""
import itertools
import math

import numpy as np

import oracle


def test_naive_digits_are_a_bijection():
    # Lemma 2: the digits of every value below the product are distinct and
    # cover every dice outcome; recombining them gives the value back
    for i, k in ((2, 1), (4, 3), (6, 5), (7, 2), (9, 3), (12, 4)):
        sizes = [i - m for m in range(k)]
        B = math.prod(sizes)
        seen = set()
        for v in range(B):
            d = oracle.naive_digits(v, i, k)
            assert all(0 <= d[m] < sizes[m] for m in range(k))
            place, back = 1, 0
            for m in range(k):  # die i - m has place value i (i-1) ... (i-m+1)
                back += d[m] * place
                place *= sizes[m]
            assert back == v
            seen.add(tuple(d))
        assert len(seen) == B


def test_single_dice_equal_the_chain_oracle():
    # with k = 1 both methods are Lemire's method on each die
    rng = np.random.default_rng(1)
    for n in (2, 3, 17, 1000, 4099):
        data = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        for seed in (0, 5, 123456789):
            a = oracle.naive_shuffle(data, seed, oracle.PAPER_NK, 1)
            b = oracle.shuffle(data, seed, oracle.PAPER_NK, 1)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _batches(n, nk, k_max):
    i = n
    while i > 1:
        k = min(oracle.k_rule(i, nk, k_max), i - 1)
        yield i, k
        i -= k


def test_same_value_as_the_chain_in_the_other_digit_order():
    # For the same batch both methods use the same attempt word and the same
    # acceptance test (leftover >= 2^64 mod B), so they draw the same value
    # v = floor(B r / 2^64): the chain's digits are its mixed-radix digits
    # most significant first (Theorem 1), the naive ones least significant
    # first.  Checked batch by batch under the paper's schedule (k up to 6)
    # and under pairs.
    for n, nk, k_max in ((1000, oracle.PAPER_NK, 6), (70001, oracle.PAPER_NK, 6),
                         (5000, oracle.NAIVE2_NK, oracle.NAIVE2_KMAX)):
        data = np.arange(n, dtype=np.uint32)
        _, jc = oracle.shuffle(data, 42, nk, k_max)
        _, jn = oracle.naive_shuffle(data, 42, nk, k_max)
        differs = False
        for i, k in _batches(n, nk, k_max):
            sizes = [i - m for m in range(k)]
            v_chain = 0
            for m in range(k):  # most significant first
                v_chain = v_chain * sizes[m] + int(jc[i - 1 - m])
            v_naive, place = 0, 1
            for m in range(k):  # least significant first
                v_naive += int(jn[i - 1 - m]) * place
                place *= sizes[m]
            assert v_chain == v_naive, (n, i, k)
            differs |= any(jc[i - 1 - m] != jn[i - 1 - m] for m in range(k))
        assert differs  # the digit orders really differ


def test_naive_shuffle_equiprobable():
    # n = 4 under pairs: the 24 permutations over 24,000 seeds, chi-square
    counts = {}
    base = np.arange(4, dtype=np.uint32)
    for seed in range(24000):
        z, _ = oracle.naive_shuffle(base, seed)
        counts[tuple(z)] = counts.get(tuple(z), 0) + 1
    assert len(counts) == 24
    chi2 = sum((c - 1000) ** 2 / 1000 for c in counts.values())
    assert chi2 < 49.7  # 23 degrees of freedom, p = 0.001


def test_naive_schedule_default_and_overflow():
    import pytest

    assert oracle.NAIVE2_NK[2] == 1 << 32 and oracle.NAIVE2_KMAX == 2
    # a schedule whose batch products can exceed the word is rejected
    with pytest.raises(RuntimeError):
        oracle.naive_shuffle(np.arange(10, dtype=np.uint32), 1, (0, 0, 1 << 32, 1 << 32, 0, 0, 0, 0, 0), 3)
