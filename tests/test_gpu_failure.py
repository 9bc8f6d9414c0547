"""Failure detection on the device, without faulting the GPU: a bounded wait
that cannot complete gives up after its limit and the host reads the status
it recorded, and a batch that runs out of attempts records BRR_ERETRY; the
context stays usable afterwards."""
import time

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


@pytest.mark.parametrize("limit_ms", [2, 20])
def test_grid_barrier_wait_times_out(brr, limit_ms):
    from paper_2408_06213_gb300._lib import BRR_ETIMEOUT

    ctx = brr.Context(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ctx.selftest_barrier_timeout(limit_ms * 1_000_000)
    dt = time.perf_counter() - t0
    assert st == BRR_ETIMEOUT
    assert limit_ms * 1e-3 <= dt < limit_ms * 1e-3 + 2.0  # gave up after its limit, not much later
    ctx.check()  # the status was read and cleared: the context is clean again
    # and still works
    data, seed = np.arange(5000, dtype=np.uint32), 17
    d = torch.from_numpy(data).cuda()
    ctx.shuffle(d, seed)
    ctx.check()
    assert np.array_equal(d.cpu().numpy().view(np.uint32), oracle.shuffle(data, seed)[0])
    ctx.close()


def test_barrier_selftest_rejects_limits_outside_range(brr):
    ctx = brr.Context(0)
    for bad in (0, 999, 100_000_001):
        with pytest.raises(brr.BrrError):
            ctx.selftest_barrier_timeout(bad)
    ctx.close()


@pytest.mark.parametrize("kind", ["fixed", "per_roll"])
def test_retry_budget_exhaustion_is_reported(brr, kind):
    """With the attempt budget lowered by the test hook, a high-rejection
    workload exhausts it and the call records BRR_ERETRY; with the default
    budget restored the same call is exact again."""
    from paper_2408_06213_gb300 import inputs
    from paper_2408_06213_gb300._lib import BRR_ERETRY

    ctx = brr.Context(0)
    b = (1 << 31) + 1
    n = 1 << 20
    if kind == "fixed":
        run = lambda: ctx.dice_fixed(b, 2, n, 5)
        ref = lambda: oracle.dice_fixed(b, 2, n, 5)
        limit = 1   # a quarter of all pairs are rejected at attempt 0
    else:
        bm1, off = inputs.dice_workload(n, seed=7)
        d_bm1, d_off = torch.from_numpy(bm1).cuda(), torch.from_numpy(off).cuda()
        run = lambda: ctx.dice(d_bm1, d_off, 5)
        ref = lambda: oracle.dice(bm1, off, 5)
        limit = 2   # about 3.5% of batches are rejected, 0.1% twice
    ctx.selftest_attempt_limit(limit)
    run()
    with pytest.raises(brr.BrrError) as ei:
        ctx.check()
    assert ei.value.status == BRR_ERETRY
    ctx.check()  # read and cleared
    ctx.selftest_attempt_limit(1 << 16)
    out = run()
    ctx.check()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref())
    with pytest.raises(brr.BrrError):
        ctx.selftest_attempt_limit(0)
    ctx.close()
