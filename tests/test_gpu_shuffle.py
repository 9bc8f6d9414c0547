"""GPU parity: batched Fisher-Yates shuffles through the C ABI against the CPU
oracle -- the swap indices j[] and the permutation, bit-exact."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", params=["chains", "rounds"])
def ctx(request):
    """A context per swap-application method: chain resolution and
    deterministic-reservation rounds must both reproduce the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2408_06213_gb300 as brr

    c = brr.Context(0)
    c.set_swap_method(c.SWAP_CHAINS if request.param == "chains" else c.SWAP_ROUNDS)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(t, dtype):
    return t.cpu().numpy().view(dtype)


def _run(ctx, data, seed, sched=None, nk=oracle.PAPER_NK, k_max=oracle.PAPER_KMAX):
    d = _dev(data)
    j = torch.empty(data.size, dtype=torch.uint32, device="cuda")
    ctx.shuffle(d, seed, sched=sched, j_out=j)
    ctx.check()
    z, jr = oracle.shuffle(data, seed, nk, k_max)
    assert np.array_equal(_np(j, np.uint32), jr)
    assert np.array_equal(_np(d, data.dtype), z)


SIZES = [0, 1, 2, 3, 4, 5, 6, 7, 8, 13, 100, 511, 512, 513, 514, 2047, 2048, 2049, 4096, 4097, 30001,
         16383, 16384, 16385, 65535, 65536, 65537, 100003]


@pytest.mark.parametrize("n", SIZES)
def test_shuffle_u32(ctx, n):
    _run(ctx, np.arange(n, dtype=np.uint32), seed=42 + n)


@pytest.mark.parametrize("n", [2, 9, 1000, 65536, 300007])
def test_shuffle_u64(ctx, n):
    rng = np.random.default_rng(n)
    _run(ctx, rng.integers(0, 1 << 63, size=n, dtype=np.uint64), seed=3)


def test_shuffle_small_config(ctx):
    from paper_2408_06213_gb300 import inputs

    data, seed = inputs.shuffle_small(65536)
    _run(ctx, data, seed)


@pytest.mark.parametrize("k_max", [1, 2, 3])
def test_shuffle_other_schedules(ctx, k_max):
    import paper_2408_06213_gb300 as brr

    _run(ctx, np.arange(70001, dtype=np.uint32), seed=9, sched=brr.schedule(k_max=k_max), k_max=k_max)


def test_shuffle_table2_schedule(ctx):
    import paper_2408_06213_gb300 as brr

    nk = (0, 0, 1358187913, 929104, 26573, 3225, 815, 305, 146)
    sched = brr.schedule({k: nk[k] for k in range(2, 9)})
    _run(ctx, np.arange(40000, dtype=np.uint32), seed=10, sched=sched, nk=nk, k_max=8)


def test_shuffle_without_j_out(ctx):
    data = np.arange(12345, dtype=np.uint32)
    d = _dev(data)
    ctx.shuffle(d, 77)
    ctx.check()
    assert np.array_equal(_np(d, np.uint32), oracle.shuffle(data, 77)[0])


def test_shuffle_repeated_calls_reuse_scratch(ctx):
    # scratch (reservations, pending lists) must be left clean between calls
    for n, seed in [(5000, 1), (300, 2), (70000, 3), (5000, 4)]:
        _run(ctx, np.arange(n, dtype=np.uint32), seed)


def test_shuffle_large_config(ctx):
    """n = 2^24 uint64 random values, seed 3: full permutation bit-exact."""
    from paper_2408_06213_gb300 import inputs

    data, seed = inputs.shuffle_large()
    _run(ctx, data, seed)


def test_shuffle_end_to_end_host_buffers(ctx):
    data = np.arange(33333, dtype=np.uint32)
    t = torch.from_numpy(data.copy())
    ctx.shuffle(t, 5)
    assert np.array_equal(t.numpy(), oracle.shuffle(data, 5)[0])
