"""GPU parity of the naive batched shuffle (the paper's division-based
comparison method) with the oracle: swap indices and permutation, bit-exact,
under both swap-application methods."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 100, 4097, 65536, 100003])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_naive_pairs(ctx, n, dtype):
    rng = np.random.default_rng(n)
    data = rng.integers(0, np.iinfo(dtype).max, size=n, dtype=dtype, endpoint=True)
    d = torch.from_numpy(data).cuda()
    j = torch.empty(max(n, 1), dtype=torch.uint32, device="cuda")
    ctx.shuffle_naive(d, 42 + n, j_out=j[:n] if n else None)
    ctx.check()
    z, jr = oracle.naive_shuffle(data, 42 + n)
    assert np.array_equal(d.cpu().numpy().view(dtype), z)
    if n:
        assert np.array_equal(j[:n].cpu().numpy().view(np.uint32), jr)


def test_naive_under_the_paper_schedule(ctx):
    # batches of up to 6 dice: products near 2^64, several divisions a batch
    import paper_2408_06213_gb300 as brr

    for n in (1000, 70001, 1 << 20):
        data = np.arange(n, dtype=np.uint32)
        d = torch.from_numpy(data).cuda()
        ctx.shuffle_naive(d, 7, sched=brr.schedule())
        ctx.check()
        z, _ = oracle.naive_shuffle(data, 7, oracle.PAPER_NK, oracle.PAPER_KMAX)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), z)


def test_naive_default_schedule_is_pairs(ctx):
    import paper_2408_06213_gb300 as brr

    s = brr.naive_schedule()
    assert s.k_max == 2 and s.n_k[2] == 1 << 32


@pytest.mark.parametrize("n", [1, 2, 65536, 1 << 20])
def test_swap_indices_only(ctx, n):
    # data NULL: only j[], for the batched, unbatched and naive methods
    import paper_2408_06213_gb300 as brr

    data = np.arange(n, dtype=np.uint32)
    for sched, ref in ((None, lambda: oracle.shuffle(data, 9)[1]),
                       (brr.schedule(k_max=1), lambda: oracle.shuffle(data, 9, oracle.PAPER_NK, 1)[1])):
        j = ctx.swap_indices(n, 9, sched=sched)
        ctx.check()
        assert np.array_equal(j.cpu().numpy().view(np.uint32), ref())
    j = ctx.swap_indices(n, 9, naive=True)
    ctx.check()
    assert np.array_equal(j.cpu().numpy().view(np.uint32), oracle.naive_shuffle(data, 9)[1])
