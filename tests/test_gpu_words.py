"""GPU parity of shuffles on the other counter-based word sources (ChaCha20 at
L = 64, the 32-bit SplitMix source with the Theorem 1 chain at L = 32) with
the oracle: swap indices and permutations bit-exact, batched and unbatched,
under both swap-application methods."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SOURCES = [("chacha20", 1), ("splitmix32", 2)]


@pytest.fixture(scope="module", params=["chains", "rounds"])
def ctx(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2408_06213_gb300 as brr

    c = brr.Context(0)
    c.set_swap_method(c.SWAP_CHAINS if request.param == "chains" else c.SWAP_ROUNDS)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx1():
    # one context with the default swap method, for the tests that do not
    # apply swaps
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2408_06213_gb300 as brr

    c = brr.Context(0)
    yield c
    c.close()


def _oracle_src(name):
    return {"chacha20": oracle.SRC_CHACHA20, "splitmix32": oracle.SRC_SPLITMIX32}[name]


@pytest.mark.parametrize("src", SOURCES, ids=[s[0] for s in SOURCES])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 7, 100, 4097, 65536, 100003])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_words_shuffle_matches_oracle(ctx, src, n, dtype):
    name, source = src
    rng = np.random.default_rng(n + 17)
    data = rng.integers(0, np.iinfo(dtype).max, size=n, dtype=dtype, endpoint=True)
    d = torch.from_numpy(data).cuda()
    j = torch.empty(max(n, 1), dtype=torch.uint32, device="cuda")
    ctx.shuffle_words(d, 1000 + n, source, j_out=j[:n] if n else None)
    ctx.check()
    z, jr = oracle.shuffle_src(_oracle_src(name), data, 1000 + n)
    assert np.array_equal(d.cpu().numpy().view(dtype), z)
    if n:
        assert np.array_equal(j[:n].cpu().numpy().view(np.uint32), jr)


@pytest.mark.parametrize("src", SOURCES, ids=[s[0] for s in SOURCES])
def test_words_unbatched_and_custom_schedules(ctx, src):
    # k_max = 1 (one word per die) and a schedule of single batches up to
    # the word size's limit
    import paper_2408_06213_gb300 as brr

    name, source = src
    n = 70001
    data = np.arange(n, dtype=np.uint32)
    base = brr.l32_schedule() if source == 2 else brr.schedule()
    nk = [int(base.n_k[k]) for k in range(9)]
    for k_max in (1, 2, int(base.k_max)):
        s = brr.l32_schedule() if source == 2 else brr.schedule()
        s.k_max = k_max
        d = torch.from_numpy(data).cuda()
        ctx.shuffle_words(d, 5, source, sched=s)
        ctx.check()
        z, _ = oracle.shuffle_src(_oracle_src(name), data, 5, nk, k_max)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), z), k_max


@pytest.mark.parametrize("src", SOURCES, ids=[s[0] for s in SOURCES])
@pytest.mark.parametrize("n", [2, 65536, 1 << 22])
def test_words_swap_indices_only(ctx, src, n):
    import paper_2408_06213_gb300 as brr

    name, source = src
    for k_max in (None, 1):
        sched = None
        kw = {}
        if k_max is not None:
            sched = brr.l32_schedule() if source == 2 else brr.schedule()
            sched.k_max = k_max
            kw = dict(nk=[int(sched.n_k[k]) for k in range(9)], k_max=k_max)
        j = ctx.swap_indices(n, 9, sched=sched, source=source)
        ctx.check()
        _, jr = oracle.shuffle_src(_oracle_src(name), None, 9, n=n, **kw)
        assert np.array_equal(j.cpu().numpy().view(np.uint32), jr)


def test_splitmix64_source_is_brr_shuffle(ctx):
    n = 5000
    data = np.arange(n, dtype=np.uint64)
    a = torch.from_numpy(data).cuda()
    b = a.clone()
    ctx.shuffle_words(a, 77, 0)
    ctx.shuffle(b, 77)
    ctx.check()
    assert torch.equal(a.view(torch.int64), b.view(torch.int64))


def test_l32_rejects_schedules_beyond_2p32(ctx):
    # the paper's L = 64 schedule forms batches whose product exceeds 2^32
    import paper_2408_06213_gb300 as brr

    d = torch.arange(1000, dtype=torch.int32, device="cuda")
    with pytest.raises(brr.BrrError):
        ctx.shuffle_words(d, 1, 2, sched=brr.schedule())
    with pytest.raises(brr.BrrError):
        ctx.shuffle_words(d, 1, 3)
    ctx.check()


def test_words_bench_sizes(ctx1):
    # the sizes the benchmark times: swap indices of an n = 2^24 shuffle with
    # ChaCha20 words (every index against the oracle), and 2^28 fixed-bound
    # rolls (b = 6, k = 6) with ChaCha20 words and at L = 32 (k = 8), sampled
    # batch by batch
    n = 1 << 24
    j = ctx1.swap_indices(n, 3, source=1)
    ctx1.check()
    _, jr = oracle.shuffle_src(oracle.SRC_CHACHA20, None, 3, n=n)
    assert np.array_equal(j.cpu().numpy().view(np.uint32), jr)
    del j
    n_d = 1 << 28
    out = torch.empty(n_d, dtype=torch.uint32, device="cuda")
    rng = np.random.default_rng(9)
    for src, k in ((oracle.SRC_CHACHA20, 6), (oracle.SRC_SPLITMIX32, 8)):
        ctx1.dice_fixed(6, k, n_d, 7, out=out, source=src)
        ctx1.check()
        got = out.cpu().numpy().view(np.uint32)
        n_b = (n_d + k - 1) // k
        for g in list(rng.integers(0, n_b, 200)) + [0, n_b - 1]:
            kk = min(k, n_d - int(g) * k)
            digits, _ = oracle.roll_batch_src(src, [6] * kk, 7, int(g))
            assert list(got[int(g) * k:int(g) * k + kk]) == digits


@pytest.mark.parametrize("src", SOURCES, ids=[s[0] for s in SOURCES])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_words_batched_shuffles_match_oracle(ctx1, src, dtype):
    # many arrays in one call on each source: every size class of the CTA
    # kernel (small, medium, large, staged and not) and the long-array kernel
    # above 65,536; each array as brr_shuffle_words would shuffle it
    name, source = src
    rng = np.random.default_rng(21)
    sizes = [0, 1, 2, 3, 16, 100, 2048, 2049, 8192, 8193, 20000, 30000, 60000, 65536, 65537, 100000]
    sizes += [int(x) for x in np.floor(16 * 4096 ** rng.random(40))]
    offsets = np.zeros(len(sizes) + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    data = rng.integers(0, np.iinfo(dtype).max, size=int(offsets[-1]), dtype=dtype, endpoint=True)
    seeds = rng.integers(0, 2**63, size=len(sizes), dtype=np.uint64)
    d = torch.from_numpy(data).cuda()
    ctx1.shuffle_batched(d, torch.from_numpy(offsets).cuda(), torch.from_numpy(seeds).cuda(), max(sizes),
                         source=source)
    ctx1.check()
    got = d.cpu().numpy().view(dtype)
    for s, n in enumerate(sizes):
        a, b = int(offsets[s]), int(offsets[s + 1])
        z, _ = oracle.shuffle_src(_oracle_src(name), data[a:b], int(seeds[s]))
        assert np.array_equal(got[a:b], z), (s, n)


@pytest.mark.parametrize("src", SOURCES, ids=[s[0] for s in SOURCES])
def test_words_batched_unbatched_schedule(ctx1, src):
    import paper_2408_06213_gb300 as brr

    name, source = src
    sizes = [5, 300, 5000, 40000]
    offsets = np.zeros(len(sizes) + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    data = np.arange(int(offsets[-1]), dtype=np.uint32)
    seeds = np.arange(1, len(sizes) + 1, dtype=np.uint64) * 977
    sched = brr.l32_schedule() if source == 2 else brr.schedule()
    sched.k_max = 1
    d = torch.from_numpy(data).cuda()
    ctx1.shuffle_batched(d, torch.from_numpy(offsets).cuda(), torch.from_numpy(seeds).cuda(), max(sizes),
                         sched=sched, source=source)
    ctx1.check()
    got = d.cpu().numpy().view(np.uint32)
    nk = [int(sched.n_k[k]) for k in range(9)]
    for s in range(len(sizes)):
        a, b = int(offsets[s]), int(offsets[s + 1])
        z, _ = oracle.shuffle_src(_oracle_src(name), data[a:b], int(seeds[s]), nk, 1)
        assert np.array_equal(got[a:b], z), s
