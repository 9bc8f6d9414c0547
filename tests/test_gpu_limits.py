"""GPU parity at the sizes the C ABI allows beyond the benchmark's: more than
2^32 fixed-bound rolls (64-bit batch and output indices) and 2^32 - 64
per-roll-bound rolls (the largest one-roll-per-batch call), checked on
sampled batches against the oracle, one batch at a time."""
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


def _gather(out, idx):
    """out[idx] for host indices idx, read back without copying all of out."""
    t = torch.from_numpy(np.asarray(idx, dtype=np.int64)).to(out.device)
    return out.view(torch.int32)[t].cpu().numpy().view(np.uint32)


def test_fixed_bound_rolls_beyond_2p32(ctx):
    # 2^32 + 1001 rolls of b = 6 in batches of 6 (16 GiB out): batches whose
    # rolls lie past index 2^32, the last (short) batch and a few early ones
    n, b, k, seed = (1 << 32) + 1001, 6, 6, 12
    out = torch.empty(n, dtype=torch.uint32, device="cuda")
    ctx.dice_fixed(b, k, n, seed, out=out)
    ctx.check()
    n_b = (n + k - 1) // k
    rng = np.random.default_rng(1)
    gs = [0, 1, (1 << 32) // k, (1 << 32) // k + 1, n_b - 2, n_b - 1] + list(rng.integers(0, n_b, 60))
    for g in gs:
        g = int(g)
        kk = min(k, n - g * k)
        got = _gather(out, range(g * k, g * k + kk))
        digits, _ = oracle.roll_batch([b] * kk, seed, g)
        assert list(got) == digits, g
    del out


def test_one_roll_per_batch_at_the_batch_limit(ctx):
    # 2^32 - 64 rolls with one roll per batch (brr_dice with no offsets): the
    # largest batch count the call takes, 32-bit batch and roll indices up to
    # their limit; one bound b = 2^31 + 1 for every roll, sampled batches up
    # to the last
    n = (1 << 32) - 64
    b = (1 << 31) + 1
    bm1 = torch.full((n,), -(1 << 31), dtype=torch.int32, device="cuda").view(torch.uint32)  # b - 1 = 2^31
    out = torch.empty(n, dtype=torch.uint32, device="cuda")
    ctx.dice(bm1, None, 5, out=out)
    ctx.check()
    rng = np.random.default_rng(2)
    gs = [0, 1, n // 2, n - 2, n - 1] + list(rng.integers(0, n, 60))
    got = _gather(out, gs)
    for g, v in zip(gs, got):
        digits, _ = oracle.roll_batch([b], 5, int(g))
        assert int(v) == digits[0], int(g)
    del bm1, out
