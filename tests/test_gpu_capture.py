"""Calls captured into a CUDA graph before brr_reserve sized the scratch.

A call whose scratch would have to grow while its stream is being captured
must return BRR_EINVAL and queue nothing, so that the caller's capture stays
valid (growing the scratch allocates and synchronises, which would
invalidate it).  Each case below runs on a fresh context, whose scratch is
empty, inside torch.cuda.graph: the BrrError must come out of the `with`
block, which means ending the capture succeeded.  The context is then used
outside the capture and checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def brr():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2408_06213_gb300 as brr

    return brr


def _capture_refused(brr, call):
    """Capture `mark += 1` then `call()`: the call must raise BRR_EINVAL and
    the capture must end cleanly, leaving a graph that replays the mark
    update alone."""
    from paper_2408_06213_gb300._lib import BRR_EINVAL

    mark = torch.zeros(1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with pytest.raises(brr.BrrError) as ei:
        with torch.cuda.graph(g, stream=side):
            mark.add_(1)
            call()
    assert ei.value.status == BRR_EINVAL
    torch.cuda.synchronize()
    assert int(mark.item()) == 0  # capturing ran nothing
    g.replay()
    torch.cuda.synchronize()
    assert int(mark.item()) == 1
    del g


def test_single_shuffle_rounds_capture_without_reserve(brr):
    ctx = brr.Context(0)
    ctx.set_swap_method(ctx.SWAP_ROUNDS)
    n, seed = 200_003, 91
    data = np.arange(n, dtype=np.uint32)
    d = torch.from_numpy(data).cuda()
    _capture_refused(brr, lambda: ctx.shuffle(d, seed))
    assert np.array_equal(d.cpu().numpy().view(np.uint32), data)  # untouched
    ctx.shuffle(d, seed)
    ctx.check()
    z, _ = oracle.shuffle(data, seed)
    assert np.array_equal(d.cpu().numpy().view(np.uint32), z)
    ctx.close()


def test_batched_shuffle_rounds_long_capture_without_reserve(brr):
    ctx = brr.Context(0)
    ctx.set_swap_method(ctx.SWAP_ROUNDS)
    sizes = np.array([40_000, 17, 33_333, 5], dtype=np.int64)
    offsets = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    rng = np.random.default_rng(5)
    data = rng.integers(0, 1 << 32, size=int(offsets[-1]), dtype=np.uint64).astype(np.uint32)
    seeds = rng.integers(0, 1 << 63, size=sizes.size, dtype=np.uint64)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(offsets).cuda()
    s = torch.from_numpy(seeds).cuda()
    _capture_refused(brr, lambda: ctx.shuffle_batched(d, o, s, int(sizes.max())))
    assert np.array_equal(d.cpu().numpy().view(np.uint32), data)
    ctx.shuffle_batched(d, o, s, int(sizes.max()))
    ctx.check()
    assert np.array_equal(d.cpu().numpy().view(np.uint32), oracle.shuffle_batched(data, offsets, seeds))
    ctx.close()


def test_sample_batched_long_capture_without_reserve(brr):
    ctx = brr.Context(0)
    n = np.array([1_000_000, 300, 70_000], dtype=np.uint64)
    m = np.array([9_000, 300, 6_001], dtype=np.uint32)
    seeds = np.array([3, 4, 5], dtype=np.uint64)
    out_off = np.zeros(4, dtype=np.uint64)
    np.cumsum(m.astype(np.uint64), out=out_off[1:])
    dn, dm = torch.from_numpy(n).cuda(), torch.from_numpy(m).cuda()
    ds, do = torch.from_numpy(seeds).cuda(), torch.from_numpy(out_off).cuda()
    out = torch.zeros(int(out_off[-1]), dtype=torch.uint32, device="cuda")
    _capture_refused(brr, lambda: ctx.sample_batched(dn, dm, ds, do, int(m.max()), out))
    assert int(out.view(torch.int32).abs().sum()) == 0
    ctx.sample_batched(dn, dm, ds, do, int(m.max()), out)
    ctx.check()
    got = out.cpu().numpy().view(np.uint32)
    for i in range(n.size):
        ref = oracle.sample(int(n[i]), int(m[i]), int(seeds[i]))
        assert np.array_equal(got[int(out_off[i]):int(out_off[i + 1])], ref)
    ctx.close()
