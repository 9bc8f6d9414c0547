"""The shuffle entry point that allocates no device memory.

brr_shuffle_noalloc exists for callers that cannot allocate device memory on
demand: their device memory belongs to another allocator or a fixed budget,
or they run latency-critical loops that cannot take the synchronisation
cudaMalloc / cudaFree may bring.  It takes its scratch from a fixed array
inside the library.  This test calls it through the C ABI and checks, on two
calls in a row, that it gives exactly what brr_shuffle gives (integer work:
bit-exact), including the swap indices and the device-side status.  The file
is collected last so that a failure here stops a -x run only after every
other test has run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

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


def _noalloc(brr, data, seed, sched=None, j_out=None, status=None):
    L = brr.lib()
    st = L.brr_shuffle_noalloc(data.data_ptr(), data.numel(), data.element_size(), seed,
                               ctypes.byref(sched) if sched is not None else None,
                               j_out.data_ptr() if j_out is not None else None,
                               status.data_ptr() if status is not None else None,
                               torch.cuda.current_stream().cuda_stream)
    return st


def test_noalloc_matches_brr_shuffle_twice(brr):
    ctx = brr.Context(0)
    rng = np.random.default_rng(2024)
    # two calls in a row: a long one, then a shorter one that must not see
    # anything the first left in the shared scratch
    for n, seed, dtype in [(300007, 11, np.uint32), (70001, 12, np.uint32)]:
        host = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(dtype)
        a = torch.from_numpy(host).cuda()
        b = a.clone()
        ja = torch.empty(n, dtype=torch.uint32, device="cuda")
        jb = torch.empty(n, dtype=torch.uint32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert _noalloc(brr, a, seed, j_out=ja, status=status) == 0
        ctx.shuffle(b, seed, j_out=jb)
        ctx.check()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
        assert torch.equal(ja.view(torch.int32), jb.view(torch.int32))
    ctx.close()


def test_noalloc_u64_without_swap_indices(brr):
    ctx = brr.Context(0)
    rng = np.random.default_rng(7)
    for n, seed in [(1 << 20, 3), (4097, 4)]:
        host = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
        a = torch.from_numpy(host).cuda()
        b = a.clone()
        assert _noalloc(brr, a, seed, sched=brr.schedule(k_max=3)) == 0
        ctx.shuffle(b, seed, sched=brr.schedule(k_max=3))
        ctx.check()
        torch.cuda.synchronize()
        assert torch.equal(a.view(torch.int64), b.view(torch.int64))
    ctx.close()


def test_noalloc_rejects_arrays_beyond_its_limit(brr):
    limit = 1 << 20
    a = torch.zeros(limit + 1, dtype=torch.uint32, device="cuda")
    assert _noalloc(brr, a, 1) == 1  # BRR_EINVAL, nothing queued
    assert int(a.view(torch.int32).abs().sum().item()) == 0
