"""Pins of the oracle's alternative word sources (ChaCha20 at L = 64, the
SplitMix64 high half at L = 32) and of the L = 32 chain and schedule, each
checked against something other than the oracle itself: a cryptographic
library's ChaCha20, the mixed-radix closed form of Theorem 1, Lemire's
32-bit method, Table 2, and uniformity over permutations."""
import math
import os

import numpy as np
import pytest

import oracle

SRCS = (oracle.SRC_SPLITMIX64, oracle.SRC_CHACHA20, oracle.SRC_SPLITMIX32)


def _library_chacha20_word(seed: int, g: int, a: int) -> int:
    """First 8 keystream bytes of the `cryptography` package's ChaCha20 with
    the key, counter and nonce of the oracle's source 1."""
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    c = (g << 16) | a
    key = seed.to_bytes(8, "little") + bytes(24)
    # the library's 16-byte nonce is the 32-bit block counter then the 96-bit nonce
    nonce = (c & 0xFFFFFFFF).to_bytes(4, "little") + (c >> 32).to_bytes(4, "little") + bytes(8)
    enc = ciphers.Cipher(ciphers.algorithms.ChaCha20(key, nonce), mode=None).encryptor()
    return int.from_bytes(enc.update(bytes(8)), "little")


def test_chacha20_words_match_library():
    rng = np.random.default_rng(11)
    cases = [(0, 0, 0), (1, 0, 1), (2**64 - 1, 2**47 - 1, 2**16 - 1), (0x0123456789ABCDEF, 12345, 3)]
    for _ in range(200):
        cases.append((int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)),
                      int(rng.integers(0, 2**40)), int(rng.integers(0, 2**16))))
    for seed, g, a in cases:
        assert oracle.word_src(oracle.SRC_CHACHA20, seed, g, a) == _library_chacha20_word(seed, g, a)


def test_chacha_block_full_keystream_matches_library():
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    seed, c = 0xDEADBEEFCAFEF00D, (987654321 << 16) | 7
    key = seed.to_bytes(8, "little") + bytes(24)
    nonce = (c & 0xFFFFFFFF).to_bytes(4, "little") + (c >> 32).to_bytes(4, "little") + bytes(8)
    ks = ciphers.Cipher(ciphers.algorithms.ChaCha20(key, nonce), mode=None).encryptor().update(bytes(64))
    out = oracle.chacha_block(oracle.chacha_input(seed, c), 20)
    assert out.astype("<u4").tobytes() == ks


def test_chacha_zero_rounds_is_input_doubled():
    # with no rounds the block function adds the input to itself
    inp = oracle.chacha_input(5, 77)
    assert np.array_equal(oracle.chacha_block(inp, 0), (inp.astype(np.uint64) * 2 % 2**32).astype(np.uint32))


def test_source_bits_and_default_source():
    assert [oracle.src_bits(s) for s in SRCS] == [64, 64, 32]
    for g, a in ((0, 0), (5, 1), (2**40, 9)):
        assert oracle.word_src(oracle.SRC_SPLITMIX64, 3, g, a) == oracle.word(3, g, a)
        assert oracle.word_src(oracle.SRC_SPLITMIX32, 3, g, a) < 2**32


def _mixed_radix_msb_first(v: int, b):
    d = []
    for bi in reversed(b):
        d.append(v % bi)
        v //= bi
    return list(reversed(d))


def test_l32_chain_closed_form():
    # Theorem 1's chain at L = 32 equals the mixed-radix digits (most
    # significant first) of floor(B r / 2^32), and leaves (B r) mod 2^32
    rng = np.random.default_rng(3)
    for _ in range(400):
        k = int(rng.integers(1, 5))
        b = []
        B = 1
        for _m in range(k):
            x = int(rng.integers(1, 2**16))
            if B * x > 2**32:
                break
            b.append(x)
            B *= x
        r0 = int(rng.integers(0, 2**32))
        a, rk = oracle.chain(32, b, r0)
        assert a == _mixed_radix_msb_first((B * r0) >> 32, b)
        assert rk == (B * r0) % 2**32


def _lemire32(s: int, seed: int, g: int) -> int:
    """Lemire's nearly-divisionless method for one 32-bit bound s, written
    out from Section 2 with the attempt words of batch g (source 2)."""
    att = 0
    m = oracle.word_src(oracle.SRC_SPLITMIX32, seed, g, att) * s
    low = m % 2**32
    if low < s:
        t = (2**32 - s) % s
        while low < t:
            att += 1
            m = oracle.word_src(oracle.SRC_SPLITMIX32, seed, g, att) * s
            low = m % 2**32
    return m >> 32


def test_l32_single_roll_is_lemire():
    rng = np.random.default_rng(8)
    bounds = [1, 2, 3, 7, 2**31, 2**31 + 1, 2**32 - 1, 3 * 2**30 + 5] + [int(x) for x in rng.integers(1, 2**32, 60)]
    for s in bounds:
        for g in range(40):
            a, _ = oracle.roll_batch_src(oracle.SRC_SPLITMIX32, [s], 21, g)
            assert a[0] == _lemire32(s, 21, g)


def test_l32_product_limit_and_full_word():
    # a batch product above 2^32 is refused at L = 32; exactly 2^32 (threshold
    # 0) accepts the first word
    with pytest.raises(oracle.OracleError):
        oracle.roll_batch_src(oracle.SRC_SPLITMIX32, [2**16 + 1, 2**16], 1, 0)
    for g in range(50):
        a, att = oracle.roll_batch_src(oracle.SRC_SPLITMIX32, [2**16, 2**16], 1, g)
        assert att == 1
        w = oracle.word_src(oracle.SRC_SPLITMIX32, 1, g, 0)
        assert a == [w >> 16, w & 0xFFFF]


def test_l32_rejection_rate():
    # b = 3 * 2^30 + 5 leaves 2^32 mod b = 2^30 - 5 rejected words: about 1/4
    b = 3 * 2**30 + 5
    words = [oracle.roll_batch_src(oracle.SRC_SPLITMIX32, [b], 4, g)[1] for g in range(4000)]
    extra = sum(w - 1 for w in words) / len(words)
    p = (2**32 % b) / 2**32
    assert abs(extra - p / (1 - p)) < 0.05


def test_l32_schedule_is_table2_rounded_down():
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_estimated_nk.txt")
    col = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        L, k, nk = (int(x) for x in line.split())
        if L == 32:
            col[k] = nk
    assert sorted(col) == [2, 3, 4] and oracle.L32_KMAX == 4
    for k, est in col.items():
        assert oracle.L32_NK[k] == 2 ** int(math.floor(math.log2(est)))
    # every batch the L = 32 schedule forms fits one 32-bit word; the L = 64
    # schedule does not
    for k in (2, 3, 4):
        assert math.prod(range(oracle.L32_NK[k] - k + 1, oracle.L32_NK[k] + 1)) <= 2**32
    with pytest.raises(oracle.OracleError):
        oracle.shuffle_src(oracle.SRC_SPLITMIX32, np.arange(10, dtype=np.uint32), 1,
                           oracle.PAPER_NK, oracle.PAPER_KMAX)


@pytest.mark.parametrize("src", SRCS)
def test_shuffle_src_is_permutation_and_swaps(src):
    for n in (0, 1, 2, 3, 17, 1000, 5000):
        data = np.arange(n, dtype=np.uint64) * 7 + 1
        z, j = oracle.shuffle_src(src, data, 99)
        assert sorted(z.tolist()) == sorted(data.tolist())
        assert all(int(j[p]) <= p for p in range(n))
        assert np.array_equal(oracle.apply_swaps(data, j), z)
        _, j2 = oracle.shuffle_src(src, None, 99, n=n)
        assert np.array_equal(j, j2)


def test_source0_is_the_default_shuffle():
    data = np.arange(3000, dtype=np.uint32)
    z0, j0 = oracle.shuffle_src(oracle.SRC_SPLITMIX64, data, 12)
    z, j = oracle.shuffle(data, 12)
    assert np.array_equal(z0, z) and np.array_equal(j0, j)


def test_sources_differ():
    data = np.arange(64, dtype=np.uint32)
    outs = [oracle.shuffle_src(s, data, 5)[0].tolist() for s in SRCS]
    assert outs[0] != outs[1] and outs[0] != outs[2] and outs[1] != outs[2]


@pytest.mark.parametrize("src", (oracle.SRC_CHACHA20, oracle.SRC_SPLITMIX32))
def test_shuffle_src_uniform_over_permutations(src):
    # n = 4: one batch of three dice (product 24) under both schedules; 4800
    # seeds, chi-square with 23 degrees of freedom (p = 0.001 critical 49.7)
    n, trials = 4, 4800
    counts = {}
    for seed in range(trials):
        z, _ = oracle.shuffle_src(src, np.arange(n, dtype=np.uint32), seed)
        key = tuple(z.tolist())
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 24
    e = trials / 24
    chi2 = sum((c - e) ** 2 / e for c in counts.values())
    assert chi2 < 49.7


@pytest.mark.parametrize("src", SRCS)
def test_dice_fixed_src_is_algorithm3_batch_by_batch(src):
    # Algorithm 2 (threshold known in advance) gives, batch by batch, what
    # Algorithm 3 (threshold formed on the rare path) gives for the same
    # words, ragged last batch included
    L = oracle.src_bits(src)
    for b, k in ((6, 5), (2**31 + 1, 1), (1000, 3 if L == 32 else 6), (2**16, 2), (3, 7)):
        n = 3 * k + 2
        out = oracle.dice_fixed_src(src, b, k, n, 17)
        for g in range((n + k - 1) // k):
            kk = min(k, n - g * k)
            digits, _ = oracle.roll_batch_src(src, [b] * kk, 17, g)
            assert list(out[g * k:g * k + kk]) == digits


def test_dice_fixed_src0_is_dice_fixed():
    for b, k in ((6, 6), (2**31 + 1, 2), (2**32, 2)):
        assert np.array_equal(oracle.dice_fixed_src(oracle.SRC_SPLITMIX64, b, k, 1001, 3),
                              oracle.dice_fixed(b, k, 1001, 3))


def test_dice_fixed_src_l32_limits_and_lemire():
    # b^k above 2^32 is refused at L = 32; single dice are Lemire's 32-bit method
    with pytest.raises(oracle.OracleError):
        oracle.dice_fixed_src(oracle.SRC_SPLITMIX32, 2**16 + 1, 2, 10, 1)
    out = oracle.dice_fixed_src(oracle.SRC_SPLITMIX32, 3 * 2**30 + 5, 1, 50, 21)
    assert list(out) == [_lemire32(3 * 2**30 + 5, 21, g) for g in range(50)]
    # b = 2^32 at L = 32: the digit is the whole word
    out = oracle.dice_fixed_src(oracle.SRC_SPLITMIX32, 2**32, 1, 20, 4)
    assert list(out) == [oracle.word_src(oracle.SRC_SPLITMIX32, 4, g, 0) for g in range(20)]


def _lemire64_src(src: int, s: int, seed: int, g: int) -> int:
    """Lemire's nearly-divisionless method (Section 2) for one bound s at L = 64
    with the attempt words of batch g of source src, written out here."""
    att = 0
    m = oracle.word_src(src, seed, g, att) * s
    low = m % 2**64
    if low < s:
        t = (2**64 - s) % s
        while low < t:
            att += 1
            m = oracle.word_src(src, seed, g, att) * s
            low = m % 2**64
    return m >> 64


def test_dice_src_unbatched_is_lemire_with_chacha_words():
    # one roll per batch (off = None): every roll is Lemire's method on the
    # ChaCha20 words of its own batch
    rng = np.random.default_rng(4)
    bounds = np.array([1, 2, 3, 2**31 + 1, 2**32 - 1, 3 * 2**30 + 5] + list(rng.integers(1, 2**32, 40)),
                      dtype=np.uint64)
    bm1 = (bounds - 1).astype(np.uint32)
    out = oracle.dice_src(oracle.SRC_CHACHA20, bm1, None, 99)
    assert list(out) == [_lemire64_src(oracle.SRC_CHACHA20, int(b), 99, g) for g, b in enumerate(bounds)]


def test_dice_src_fixed_batches_match_algorithm2():
    # batches of one repeated bound: Algorithm 3 (per-roll bounds) gives what
    # Algorithm 2 (threshold known in advance) gives, for every source
    for src in SRCS:
        L = oracle.src_bits(src)
        b, k = (1000, 3) if L == 32 else (1000, 6)
        n = 10 * k + 1
        bm1 = np.full(n, b - 1, dtype=np.uint32)
        off = np.array(list(range(0, n, k)) + [n], dtype=np.uint32)
        assert np.array_equal(oracle.dice_src(src, bm1, off, 5), oracle.dice_fixed_src(src, b, k, n, 5))


def test_dice_src0_is_dice():
    from paper_2408_06213_gb300 import inputs

    bm1, off = inputs.dice_workload(5000, seed=3)
    assert np.array_equal(oracle.dice_src(oracle.SRC_SPLITMIX64, bm1, off, 8), oracle.dice(bm1, off, 8))
