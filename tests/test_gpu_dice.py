"""GPU parity: bulk batched dice through the C ABI against the CPU oracle,
bit-exact (all arithmetic is exact integer work)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2408_06213_gb300 as brr

    c = brr.Context(0)
    yield c
    c.close()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [1, 2, 5, 1000, 1023, 1024, 1025, 8191, 8192, 8193, 100003, 1 << 20])
def test_dice_var_csr(ctx, n):
    from paper_2408_06213_gb300 import inputs

    bm1, off = inputs.dice_workload(n, seed=7 + n)
    out = ctx.dice(_dev(bm1), _dev(off), seed=n)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice(bm1, off, n))


@pytest.mark.parametrize("n", [1, 7, 8191, 8192, 8193, 300001])
def test_dice_unbatched(ctx, n):
    from paper_2408_06213_gb300 import inputs

    bm1 = inputs.dice_bounds(n, seed=11)
    out = ctx.dice(_dev(bm1), None, seed=5)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice(bm1, None, 5))


@pytest.mark.parametrize("b,k", [(6, 6), (52, 6), (1000, 6), ((1 << 31) + 1, 2), (1, 5), (2, 64),
                                 (1 << 32, 2), (1 << 32, 1), (3, 40), ((1 << 32) - 1, 1), (6, 1), (7, 3)])
@pytest.mark.parametrize("n", [1, 9, 8190, 65537, 250001])
def test_dice_fixed(ctx, b, k, n):
    out = ctx.dice_fixed(b, k, n, seed=7)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_fixed(b, k, n, 7))


def test_dice_edge_bounds(ctx):
    # bounds of 1 (digit always 0), 2^32, and batches whose product is exactly 2^64
    bm1 = np.array([0, 0xFFFFFFFF, 0xFFFFFFFF, 0, 5, 0xFFFFFFFF, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,
                    0, 0xFFFF, 0xFFFF, 0xFFFFFFFF], dtype=np.uint32)
    off = np.array([0, 1, 3, 4, 6, 20, 24], dtype=np.uint32)
    out = ctx.dice(_dev(bm1), _dev(off), seed=3)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice(bm1, off, 3))


def test_dice_long_batches_unstaged(ctx):
    # a tile with more than 8192 rolls (many dice of bound 1) takes the global path
    n = 30000
    bm1 = np.zeros(n, dtype=np.uint32)
    bm1[[0, 5000, 9000, 10000, 24999, 26000]] = [12345, 77, 7, 99, 3, 5]
    off = np.array([0, 9000, 9001, 25000, n], dtype=np.uint32)
    out = ctx.dice(_dev(bm1), _dev(off), seed=8)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice(bm1, off, 8))


def test_dice_empty_batches(ctx):
    bm1 = np.array([5, 6, 7], dtype=np.uint32)
    off = np.array([0, 0, 2, 2, 3, 3], dtype=np.uint32)
    out = ctx.dice(_dev(bm1), _dev(off), seed=1)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice(bm1, off, 1))


def test_dice_invalid_product_is_reported(ctx):
    from paper_2408_06213_gb300 import BrrError

    bm1 = np.array([0xFFFFFFFF, 0xFFFFFFFF, 2], dtype=np.uint32)  # 2^32 * 2^32 * 3 > 2^64
    off = np.array([0, 3], dtype=np.uint32)
    ctx.dice(_dev(bm1), _dev(off), seed=1)
    with pytest.raises(BrrError) as e:
        ctx.check()
    assert e.value.status == 1
    ctx.check()  # the error word is cleared after it is read


def test_dice_bad_offsets_are_reported(ctx):
    from paper_2408_06213_gb300 import BrrError

    bm1 = np.arange(10, dtype=np.uint32)
    off = np.array([0, 5, 3, 10], dtype=np.uint32)
    ctx.dice(_dev(bm1), _dev(off), seed=1)
    with pytest.raises(BrrError):
        ctx.check()


def test_dice_host_arguments_rejected(ctx):
    from paper_2408_06213_gb300 import BrrError

    with pytest.raises(BrrError):
        ctx.dice_fixed(7, 23, 10, 1)  # 7^23 > 2^64
    with pytest.raises(BrrError):
        ctx.dice_fixed(0, 1, 10, 1)
    with pytest.raises(BrrError):
        ctx.dice_fixed((1 << 32) + 1, 1, 10, 1)


def test_dice_end_to_end_host_buffers(ctx):
    from paper_2408_06213_gb300 import inputs

    bm1, off = inputs.dice_workload(50000, seed=2)
    out = ctx.dice(torch.from_numpy(bm1), torch.from_numpy(off), seed=4)
    assert not out.is_cuda
    assert np.array_equal(out.numpy().view(np.uint32), oracle.dice(bm1, off, 4))


def test_dice_full_size_whole(ctx):
    """2^30 rolls with per-roll log-uniform bounds (the bulk-dice workload),
    then 2^30 rolls for each fixed bound, in the launch configuration the
    benchmark times; every roll compared with the oracle (run on all host
    cores over batch ranges, which the counter-based words allow)."""
    from paper_2408_06213_gb300 import inputs

    n = 1 << 30
    bm1, off = inputs.dice_workload(n, seed=7)
    d_bm1, d_off = _dev(bm1), _dev(off)
    out = ctx.dice(d_bm1, d_off, seed=7)
    ctx.check()
    got = _u32(out)
    del d_bm1, d_off, out
    ref = oracle.dice_parallel(bm1, off, 7)
    assert np.array_equal(got, ref)
    del got, ref, bm1, off
    for b in inputs.FIXED_BOUNDS:
        k = inputs.fixed_k(b)
        out = ctx.dice_fixed(b, k, n, seed=7)
        ctx.check()
        got = _u32(out)
        del out
        assert np.array_equal(got, oracle.dice_fixed_parallel(b, k, n, 7)), b
        del got


def test_threshold_routine_exact(ctx):
    """The device's rare-path threshold 2^64 mod B against exact integer
    arithmetic, over every magnitude class the routine distinguishes."""
    import paper_2408_06213_gb300 as brr

    import random

    rnd = random.Random(5)
    B = [1, 2, 3, 5, 7, (1 << 62) - 1, 1 << 62, (1 << 62) + 1, (1 << 63) - 1, 1 << 63, (1 << 63) + 1,
         (1 << 64) - 1, 0x5555555555555555, 0x5555555555555556, 6148914691236517203]
    for s in range(0, 64):
        lo, hi = 1 << (63 - s), (1 << (64 - s)) - 1
        B += [lo, lo + 1, hi, max(lo, hi - 1)] + [rnd.randint(lo, hi) for _ in range(400)]
    B = np.array(B, dtype=np.uint64)
    d_B = torch.from_numpy(B).cuda()
    d_t = torch.empty_like(d_B)
    st = brr.lib().brr_selftest_threshold(d_B.data_ptr(), d_t.data_ptr(), B.size,
                                          torch.cuda.current_stream().cuda_stream)
    assert st == 0
    got = d_t.cpu().numpy()
    for b, t in zip(B.tolist(), got.tolist()):
        assert t == (1 << 64) % b, b


# bounds and batch sizes with high, medium and negligible rejection rates,
# full-word bounds (b = 2^32) and every unrolled batch size
FIXED_CASES = [((1 << 31) + 1, 2), (1000, 6), (3 * (1 << 30) + 5, 1), (5, 8), (1 << 32, 2), (1 << 32, 1),
               (2**21 + 7, 3), (65521, 4), (6, 7), (11, 5)]


@pytest.mark.parametrize("b,k", FIXED_CASES)
@pytest.mark.parametrize("n", [1, 3, 31, 4097, 65537, 1000003, 1 << 22])
def test_dice_fixed_sweep_and_tiles_agree_with_oracle(ctx, b, k, n):
    # both fixed-bound kernels (sweep and tiled) give the oracle's rolls bit
    # for bit, ragged tails included
    ref = oracle.dice_fixed(b, k, n, 11)
    try:
        for mode in (0, 1):
            ctx.tune(ctx.TUNE_FIXED_SWEEP, mode)
            out = ctx.dice_fixed(b, k, n, seed=11)
            ctx.check()
            assert np.array_equal(_u32(out), ref), mode
    finally:
        ctx.tune(ctx.TUNE_FIXED_SWEEP, 1)


def test_fixed_sweep_tune_values(ctx):
    from paper_2408_06213_gb300 import BrrError

    assert ctx.tune_get(ctx.TUNE_FIXED_SWEEP) == 1
    with pytest.raises(BrrError):
        ctx.tune(ctx.TUNE_FIXED_SWEEP, 2)


# fixed-bound dice on the other word sources (ChaCha20 at L = 64, the 32-bit
# SplitMix source at L = 32): bit-exact against the oracle's Algorithm 2
L32_CASES = [(6, 6), (6, 8), (1000, 3), (3 * (1 << 30) + 5, 1), (1 << 16, 2), (65521, 2), (11, 5), (3, 7),
             (1 << 32, 1)]
L64_CASES = L32_CASES + [((1 << 31) + 1, 2), (1000, 6), (1 << 32, 2)]


@pytest.mark.parametrize("src,b,k", [(1, b, k) for b, k in L64_CASES] + [(2, b, k) for b, k in L32_CASES])
@pytest.mark.parametrize("n", [1, 33, 4097, 100003, 1 << 20])
def test_dice_fixed_words_match_oracle(ctx, src, b, k, n):
    out = ctx.dice_fixed(b, k, n, seed=23, source=src)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_fixed_src(src, b, k, n, 23))


@pytest.mark.parametrize("src", [1, 2])
def test_dice_fixed_words_unaligned_output(ctx, src):
    # an output that is not 16-byte aligned takes the one-thread-per-batch kernel
    n = 50001
    buf = torch.empty(n + 1, dtype=torch.uint32, device="cuda")
    out = buf[1:]
    ctx.dice_fixed(6, 5, n, seed=2, out=out, source=src)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_fixed_src(src, 6, 5, n, 2))


def test_dice_fixed_words_argument_errors(ctx):
    from paper_2408_06213_gb300 import BrrError

    for src, b, k in ((2, 1 << 16 | 1, 2), (2, 6, 9), (1, 6, 9), (3, 6, 2), (1, 0, 1), (2, (1 << 32) + 1, 1)):
        with pytest.raises(BrrError):
            ctx.dice_fixed(b, k, 10, seed=1, source=src)
    # source 0 keeps brr_dice_fixed's wider k
    out = ctx.dice_fixed(2, 64, 100, seed=1, source=0)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_fixed(2, 64, 100, 1))


def test_dice_host_buffers_on_two_streams_without_sync(ctx):
    # host-buffer calls queued on two streams (sync=False) overlap their
    # copies and keep separate staging buffers; results match the oracle
    from paper_2408_06213_gb300 import inputs

    bm1, off = inputs.dice_workload(300000, seed=5)
    n = bm1.size
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    out_a = torch.empty(n, dtype=torch.uint32, pin_memory=True)
    out_b = torch.empty(n, dtype=torch.uint32, pin_memory=True)
    out_c = torch.empty(n, dtype=torch.uint32, pin_memory=True)
    ctx.dice(torch.from_numpy(bm1).pin_memory(), torch.from_numpy(off).pin_memory(), 8, out=out_a,
             stream=sa, sync=False)
    ctx.dice_fixed(1000, 6, n, 8, out=out_b, stream=sb, sync=False)
    ctx.dice_fixed((1 << 31) + 1, 2, n, 9, out=out_c, stream=sb, sync=False)
    ctx.check(sa)
    ctx.check(sb)
    assert np.array_equal(out_a.numpy().view(np.uint32), oracle.dice(bm1, off, 8))
    assert np.array_equal(out_b.numpy().view(np.uint32), oracle.dice_fixed(1000, 6, n, 8))
    assert np.array_equal(out_c.numpy().view(np.uint32), oracle.dice_fixed((1 << 31) + 1, 2, n, 9))


def _l32_workload(n, seed):
    """Bounds log-uniform on [2, 2^20], grouped greedily into batches of up to
    8 whose product stays at most 2^32 (the L = 32 counterpart of the bulk
    workload's grouping)."""
    rng = np.random.default_rng(seed)
    b = np.floor(2.0 ** (1 + 19 * rng.random(n))).astype(np.uint64)
    off, prod, k = [0], 1, 0
    for x, bx in enumerate(b):
        if k == 8 or prod * int(bx) > 1 << 32:
            off.append(x)
            prod, k = 1, 0
        prod *= int(bx)
        k += 1
    off.append(n)
    return (b - 1).astype(np.uint32), np.array(off, dtype=np.uint32)


@pytest.mark.parametrize("n", [1, 33, 4097, 100003, 1 << 20])
def test_dice_words_per_roll_bounds_match_oracle(ctx, n):
    # per-roll bounds (Algorithm 3) on the ChaCha20 words (the bulk workload's
    # batches) and at L = 32 (batches grouped to products <= 2^32), batched and
    # one roll per batch
    from paper_2408_06213_gb300 import inputs

    bm1, off = inputs.dice_workload(n, seed=n + 3)
    out = ctx.dice(_dev(bm1), _dev(off), seed=31, source=1)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_src(1, bm1, off, 31))
    out = ctx.dice(_dev(bm1), None, seed=31, source=1)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_src(1, bm1, None, 31))
    bm1, off = _l32_workload(n, n + 5)
    out = ctx.dice(_dev(bm1), _dev(off), seed=32, source=2)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_src(2, bm1, off, 32))
    out = ctx.dice(_dev(bm1), None, seed=32, source=2)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_src(2, bm1, None, 32))


def test_dice_words_l32_products_and_full_words(ctx):
    # at L = 32 a batch product above 2^32 is reported on the device; b = 2^32
    # as a single die, and two dice of 2^16 (product exactly 2^32), accept the
    # first word
    from paper_2408_06213_gb300 import BrrError

    bm1 = np.array([0xFFFF, 0xFFFF, 0xFFFFFFFF, 0xFFFF, 0xFFFF, 6], dtype=np.uint32)
    off = np.array([0, 2, 3, 6], dtype=np.uint32)  # last batch 2^16 * 2^16 * 7 > 2^32
    ctx.dice(_dev(bm1), _dev(off), seed=1, source=2)
    with pytest.raises(BrrError):
        ctx.check()
    off = np.array([0, 2, 3, 5, 6], dtype=np.uint32)
    out = ctx.dice(_dev(bm1), _dev(off), seed=1, source=2)
    ctx.check()
    assert np.array_equal(_u32(out), oracle.dice_src(2, bm1, off, 1))
    with pytest.raises(BrrError):
        ctx.dice(_dev(bm1), _dev(off), seed=1, source=3)



@pytest.mark.parametrize("n", [3, 4, 257, 1029, 70001, (1 << 22) + 5])
def test_dice_var_unaligned_bounds(ctx, n):
    # bm1 and out not 16-byte aligned (views one element into their buffers)
    from paper_2408_06213_gb300 import inputs

    bm1, off = inputs.dice_workload(n, seed=3 + n)
    buf = torch.empty(bm1.size + 1, dtype=torch.uint32, device="cuda")
    buf[1:].copy_(_dev(bm1))
    obuf = torch.empty(bm1.size + 1, dtype=torch.uint32, device="cuda")
    ctx.dice(buf[1:], _dev(off), seed=9, out=obuf[1:])
    ctx.check()
    assert np.array_equal(_u32(obuf[1:]), oracle.dice(bm1, off, 9))


def test_dice_long_batches_on_the_exact_path(ctx):
    # batches of more than 255 dice whose product is close to 2^64 (256 dice
    # of bound 1, then 2^32 and 2^31 + 1): about half their words are
    # rejected, so they go through the pending queue of the exact test,
    # which must keep their full dice count
    reps = 300
    one = np.concatenate([np.zeros(256, dtype=np.uint32),
                          np.array([0xFFFFFFFF, 0x80000000], dtype=np.uint32)])
    bm1 = np.concatenate([one] * reps + [np.array([4, 5, 6], dtype=np.uint32)])
    off = np.concatenate([np.arange(reps + 1, dtype=np.uint32) * one.size,
                          np.array([bm1.size], dtype=np.uint32)])
    for seed in (1, 2, 3):
        out = ctx.dice(_dev(bm1), _dev(off), seed=seed)
        ctx.check()
        assert np.array_equal(_u32(out), oracle.dice(bm1, off, seed)), seed
