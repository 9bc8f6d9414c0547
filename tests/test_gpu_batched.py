"""GPU parity: many independent shuffles in one launch and partial
Fisher-Yates samples, through the C ABI, bit-exact against the CPU oracle."""
import numpy as np
import pytest

import oracle
from _sample_ref import sample_sparse

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", params=["chains", "chains_only", "rounds"])
def ctx(request):
    """A context per swap-application method: chain resolution (with the
    small and staged large arrays routed to reservation windows, and
    without), and deterministic-reservation rounds, must all reproduce the
    oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2408_06213_gb300 as brr

    c = brr.Context(0)
    c.set_swap_method(c.SWAP_ROUNDS if request.param == "rounds" else c.SWAP_CHAINS)
    c.tune(c.TUNE_WINDOW_ROUTE, 0 if request.param == "chains_only" else 1)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run_batched(ctx, sizes, dtype, seed=1, max_len=None, sched=None, nk=oracle.PAPER_NK,
                 k_max=oracle.PAPER_KMAX):
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    info = np.iinfo(dtype)
    data = rng.integers(0, info.max, size=int(offsets[-1]), dtype=dtype, endpoint=True)
    seeds = rng.integers(0, 1 << 63, size=sizes.size, dtype=np.uint64)
    d = _dev(data)
    ml = int(sizes.max()) if max_len is None else max_len
    ctx.shuffle_batched(d, _dev(offsets), _dev(seeds), ml, sched=sched)
    ctx.check()
    ref = oracle.shuffle_batched(data, offsets, seeds, nk, k_max)
    assert np.array_equal(d.cpu().numpy().view(dtype), ref)


def test_batched_small_mixed_sizes(ctx):
    sizes = [0, 1, 2, 3, 7, 16, 100, 511, 512, 513, 2047, 2049, 4097, 16384, 16385, 20000]
    _run_batched(ctx, sizes, np.uint32)
    _run_batched(ctx, sizes, np.uint64)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_batched_arrays_beyond_shared_memory(ctx, dtype):
    # arrays longer than the shared-memory staging capacity use global scratch
    _run_batched(ctx, [65536, 30000, 100, 40001, 5, 65536, 23000, 17000], dtype, seed=2)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_batched_arrays_beyond_cluster_capacity(ctx, dtype):
    # arrays longer than a cluster's shared memory are shuffled in place with
    # per-CTA global scratch
    _run_batched(ctx, [100000, 70001, 5, 65537, 65536, 3000], dtype, seed=5)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_batched_tier_boundaries(ctx, dtype):
    # lengths around where one CTA's shared memory ends (about 28,800 4-byte
    # or 19,200 8-byte elements), where a cluster's ends (65,536) and the
    # smallest arrays, so every kernel and each side of each boundary runs
    sizes = (list(range(28700, 28950, 50)) + list(range(19100, 19350, 50)) +
             [65535, 65536, 65537, 2, 3, 4096, 4097])
    _run_batched(ctx, sizes, dtype, seed=11)


def test_batched_many_arrays_log_uniform(ctx):
    from paper_2408_06213_gb300 import inputs

    data, offsets, seeds, max_len = inputs.batched_shuffles(3000, seed=4)
    d = _dev(data)
    ctx.shuffle_batched(d, _dev(offsets), _dev(seeds), max_len)
    ctx.check()
    assert np.array_equal(d.cpu().numpy().view(np.uint32), oracle.shuffle_batched(data, offsets, seeds))


def test_batched_unbatched_schedule(ctx):
    import paper_2408_06213_gb300 as brr

    _run_batched(ctx, [1000, 3, 30000, 64], np.uint32, seed=3, sched=brr.schedule(k_max=1), k_max=1)


def test_batched_rejects_long_array(ctx):
    from paper_2408_06213_gb300 import BrrError

    sizes = np.array([10, 300, 20], dtype=np.int64)
    offsets = np.zeros(4, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    data = np.arange(330, dtype=np.uint32)
    d = _dev(data)
    ctx.shuffle_batched(d, _dev(offsets), _dev(np.arange(3, dtype=np.uint64)), 100)
    with pytest.raises(BrrError):
        ctx.check()
    out = d.cpu().numpy().view(np.uint32)
    assert np.array_equal(out[10:310], data[10:310])  # the long array is untouched


def test_batched_full_config_whole(ctx):
    """65,536 arrays with log-uniform sizes in [16, 65,536] (5.2e8 uint32
    elements), in the launch configuration the benchmark times: every array
    compared element by element with the oracle (run on all host cores over
    arrays)."""
    from paper_2408_06213_gb300 import inputs

    data, offsets, seeds, max_len = inputs.batched_shuffles()
    d = _dev(data)
    ctx.shuffle_batched(d, _dev(offsets), _dev(seeds), max_len)
    ctx.check()
    got = d.cpu().numpy().view(np.uint32)
    del d
    assert np.array_equal(got, oracle.shuffle_batched_parallel(data, offsets, seeds))


# ---------------------------------------------------------------- samples --
SAMPLE_CASES = [(1, 1), (2, 1), (2, 2), (5, 5), (5, 4), (6, 3), (100, 0), (100, 1), (100, 100),
                (100, 99), (1000, 7), (513, 512), (65536, 1000), (10 ** 7, 1), (10 ** 7, 10000),
                (10 ** 7, 9999), (12345, 12345), (3000000, 4096), (2 ** 32 - 1, 77)]


@pytest.mark.parametrize("n,m", SAMPLE_CASES)
def test_sample_single(ctx, n, m):
    out = ctx.sample(n, m, seed=n + 31 * m)
    ctx.check()
    got = out.cpu().numpy().view(np.uint32)
    if n > 10 ** 8:
        # the oracle materialises n: compare with the sparse restatement
        assert np.array_equal(got, sample_sparse(n, m, n + 31 * m))
    else:
        assert np.array_equal(got, oracle.sample(n, m, n + 31 * m))


def test_sample_large_m_global_scratch(ctx):
    # m above the shared-memory capacity of one CTA
    for n, m in [(10 ** 6, 20000), (30000, 30000), (70000, 65000)]:
        out = ctx.sample(n, m, seed=m)
        ctx.check()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.sample(n, m, m))


def test_sample_batched_mixed(ctx):
    from paper_2408_06213_gb300 import inputs

    t, kind, n, m, seeds = inputs.serving_trace(400, seed=6)
    sel = kind == 1
    n, m, seeds = n[sel], m[sel], seeds[sel]
    out_off = np.zeros(n.size + 1, dtype=np.uint64)
    np.cumsum(m, out=out_off[1:])
    out = torch.empty(int(out_off[-1]), dtype=torch.uint32, device="cuda")
    ctx.sample_batched(_dev(n.astype(np.uint64)), _dev(m.astype(np.uint32)), _dev(seeds),
                       _dev(out_off[:-1].copy()), int(m.max()), out)
    ctx.check()
    got = out.cpu().numpy().view(np.uint32)
    for r in range(n.size):
        a, b = int(out_off[r]), int(out_off[r + 1])
        assert np.array_equal(got[a:b], oracle.sample(int(n[r]), int(m[r]), int(seeds[r]))), r


def test_sample_equals_shuffle_tail(ctx):
    # sample(n, n) is the full shuffle of the identity read from the top
    n = 4099
    out = ctx.sample(n, n, seed=11)
    ctx.check()
    z, _ = oracle.shuffle(np.arange(n, dtype=np.uint32), 11)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), z[::-1])


def test_window_route_tune_values(ctx):
    from paper_2408_06213_gb300 import BrrError

    with pytest.raises(BrrError):
        ctx.tune(ctx.TUNE_WINDOW_ROUTE, 2)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_batched_window_route_boundaries(ctx, dtype):
    # both sides of every routing boundary: the small class (2,048), the
    # medium class (8,192), the largest arrays the 256-thread windows class
    # stages (8,016 4-byte or 4,808 8-byte elements), the 512-thread one
    # (17,744 or 10,646), the 1024-thread one (37,072 or 22,242), the
    # 1024-thread one with the targets in global memory (55,608 or 27,804),
    # and the 16-bit limit
    sizes = ([2, 3, 127, 128, 129, 1023, 1024, 1025, 2047, 2048, 2049, 8191, 8192, 8193, 8194] +
             list(range(37020, 37130, 10)) + list(range(22200, 22300, 10)) + list(range(17700, 17800, 10)) +
             list(range(10620, 10680, 5)) +
             [4808, 4809, 8016, 8017, 10646, 10647, 17744, 17745, 22242, 22243, 37072, 37073] +
             [27804, 27805, 55608, 55609] + list(range(27780, 27830, 10)) + list(range(55580, 55640, 10)) +
             list(range(4790, 4830, 5)) + list(range(7990, 8040, 5)) +
             [13648, 16376, 27512, 35704, 41272, 65535, 65536])
    _run_batched(ctx, sizes, dtype, seed=23)
