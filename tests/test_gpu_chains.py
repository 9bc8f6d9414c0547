"""GPU parity of every kernel route of the chain-resolution shuffles.

Which kernel applies a shuffle's swaps depends on the array length and on the
context's routing parameters (brr_tune): one CTA of a size class (elements
staged in shared memory, or gathered from a global copy with part of the
links in global memory too), the grid-wide passes (one cooperative launch or
one launch per pass), or one CTA per array in global memory for long batched
arrays.  Each route is forced here over lengths on both sides of its limits
and compared with the oracle bit for bit (swap indices and permutation)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def brr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2408_06213_gb300 as brr

    return brr


def _ctx(brr, cta_max, cooperative=1):
    c = brr.Context(0)
    c.set_swap_method(c.SWAP_CHAINS)
    c.tune(c.TUNE_SINGLE_CTA_MAX, cta_max)
    c.tune(c.TUNE_GRID_COOPERATIVE, cooperative)
    return c


ROUTES = {"cta": (65536,), "grid": (0,), "grid-per-pass": (0, 0)}
SIZES = [2, 3, 7, 100, 4097, 19000, 20000, 29000, 30001, 50000, 57000, 65535, 65536]
LONG = [65537, 300007]  # grid routes only


@pytest.mark.parametrize("route", list(ROUTES))
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_single_array_routes(brr, route, dtype):
    ctx = _ctx(brr, *ROUTES[route])
    rng = np.random.default_rng(7)
    for n in SIZES + (LONG if route.startswith("grid") else []):
        data = rng.integers(0, np.iinfo(dtype).max, size=n, dtype=dtype, endpoint=True)
        d = torch.from_numpy(data).cuda()
        j = torch.empty(n, dtype=torch.uint32, device="cuda")
        ctx.shuffle(d, 1000 + n, j_out=j)
        ctx.check()
        z, jr = oracle.shuffle(data, 1000 + n)
        assert np.array_equal(j.cpu().numpy().view(np.uint32), jr), (route, n)
        assert np.array_equal(d.cpu().numpy().view(dtype), z), (route, n)
    ctx.close()


@pytest.mark.parametrize("ordered", [0, 1])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_batched_routes(brr, dtype, ordered):
    # ordered = 1: the CTA kernels roll their batches in barrier-separated
    # rounds (BRR_TUNE_ORDERED_PUSH); the result must not change
    ctx = _ctx(brr, 4096)
    ctx.tune(ctx.TUNE_ORDERED_PUSH, ordered)
    sizes = np.array([65536, 5, 30001, 57000, 60000, 19000, 100, 70001, 2, 65535, 45000, 131072],
                     dtype=np.int64)
    offsets = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    rng = np.random.default_rng(3)
    data = rng.integers(0, np.iinfo(dtype).max, size=int(offsets[-1]), dtype=dtype, endpoint=True)
    seeds = rng.integers(0, 1 << 63, size=sizes.size, dtype=np.uint64)
    d = torch.from_numpy(data).cuda()
    ctx.shuffle_batched(d, torch.from_numpy(offsets).cuda(), torch.from_numpy(seeds).cuda(), int(sizes.max()))
    ctx.check()
    assert np.array_equal(d.cpu().numpy().view(dtype), oracle.shuffle_batched(data, offsets, seeds))
    ctx.close()


def test_tune_rejects_unknown(brr):
    ctx = brr.Context(0)
    with pytest.raises(brr.BrrError):
        ctx.tune(99, 1)
    with pytest.raises(brr.BrrError):
        ctx.tune(ctx.TUNE_GRID_COOPERATIVE, 2)
    with pytest.raises(brr.BrrError):
        ctx.tune(ctx.TUNE_SMALL_MAX, 65537)
    with pytest.raises(brr.BrrError):
        ctx.tune(ctx.TUNE_ORDERED_PUSH, 2)
    ctx.tune(ctx.TUNE_SINGLE_CTA_MAX, 123)
    assert ctx.tune_get(ctx.TUNE_SINGLE_CTA_MAX) == 123
    with pytest.raises(brr.BrrError):
        ctx.set_swap_method(3)
    ctx.close()


@pytest.mark.parametrize("small_max,medium_max", [(2048, 8192), (0, 0), (65536, 65536), (100, 30000)])
def test_batched_size_classes(brr, small_max, medium_max):
    # the size-class limits move arrays between the 128-, 256- and
    # 1024-thread CTA kernels (limits above what fits one CTA are clamped)
    ctx = _ctx(brr, 4096)
    ctx.tune(ctx.TUNE_SMALL_MAX, small_max)
    ctx.tune(ctx.TUNE_MEDIUM_MAX, medium_max)
    sizes = np.array([2, 99, 100, 101, 2047, 2048, 2049, 8191, 8192, 8193, 28000, 30000, 30001,
                      57000, 65536, 16, 3], dtype=np.int64)
    offsets = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    rng = np.random.default_rng(small_max + medium_max)
    for dtype in (np.uint32, np.uint64):
        data = rng.integers(0, np.iinfo(dtype).max, size=int(offsets[-1]), dtype=dtype, endpoint=True)
        seeds = rng.integers(0, 1 << 63, size=sizes.size, dtype=np.uint64)
        d = torch.from_numpy(data).cuda()
        ctx.shuffle_batched(d, torch.from_numpy(offsets).cuda(), torch.from_numpy(seeds).cuda(), int(sizes.max()))
        ctx.check()
        assert np.array_equal(d.cpu().numpy().view(dtype), oracle.shuffle_batched(data, offsets, seeds))
    ctx.close()


@pytest.mark.parametrize("method", ["chains", "rounds"])
def test_batched_shuffle_in_a_cuda_graph(brr, method):
    """The batched launch captured once into a CUDA graph and replayed: each
    replay shuffles the arrays again, exactly as a direct call would."""
    from paper_2408_06213_gb300 import inputs

    ctx = brr.Context(0)
    ctx.set_swap_method(ctx.SWAP_CHAINS if method == "chains" else ctx.SWAP_ROUNDS)
    data, offsets, seeds, max_len = inputs.batched_shuffles(1500, seed=8)
    ctx.reserve(max_len)  # no allocation may happen while capturing
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(offsets).cuda()
    s = torch.from_numpy(seeds).cuda()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # first call outside the capture (kernel setup)
        ctx.shuffle_batched(d, o, s, max_len)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    ctx.check()
    once = oracle.shuffle_batched(data, offsets, seeds)
    assert np.array_equal(d.cpu().numpy().view(np.uint32), once)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.shuffle_batched(d, o, s, max_len)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy().view(np.uint32), once)  # capture runs nothing
    g.replay()
    torch.cuda.synchronize()
    ctx.check()
    twice = oracle.shuffle_batched(once, offsets, seeds)
    assert np.array_equal(d.cpu().numpy().view(np.uint32), twice)
    g.replay()
    torch.cuda.synchronize()
    ctx.check()
    assert np.array_equal(d.cpu().numpy().view(np.uint32), oracle.shuffle_batched(twice, offsets, seeds))
    del g
    ctx.close()
