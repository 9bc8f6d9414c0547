"""The autotuner on the GPU: it only changes routing (outputs stay equal to
the oracle's), and the schedule it suggests reproduces the oracle with that
schedule."""
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


def test_tune_batched_then_shuffle(brr):
    from paper_2408_06213_gb300 import inputs, tune

    ctx = brr.Context(0)
    data, offsets, seeds, max_len = inputs.batched_shuffles(2000, seed=12)
    res = tune.tune_batched(ctx, offsets, max_len, reps=1, passes=1)
    assert res.settings["small_max"] in tune.SMALL_MAX and res.settings["medium_max"] in tune.MEDIUM_MAX
    assert tune.current(ctx)["small_max"] == res.settings["small_max"]
    d = torch.from_numpy(data).cuda()
    ctx.shuffle_batched(d, torch.from_numpy(offsets).cuda(), torch.from_numpy(seeds).cuda(), max_len)
    ctx.check()
    assert np.array_equal(d.cpu().numpy().view(np.uint32), oracle.shuffle_batched(data, offsets, seeds))
    ctx.close()


def test_tune_single_then_shuffle(brr):
    from paper_2408_06213_gb300 import tune

    ctx = brr.Context(0)
    res = tune.tune_single(ctx, sizes=(1024, 4096, 16384), reps=2, large=1 << 20)
    assert res.settings["grid_cooperative"] in (0, 1)
    assert res.settings["single_cta_max"] in (0, 1024, 4096, 16384)
    for n in (3000, 20000, 70001):
        a = np.arange(n, dtype=np.uint32)
        d = torch.from_numpy(a).cuda()
        ctx.shuffle(d, n)
        ctx.check()
        assert np.array_equal(d.cpu().numpy().view(np.uint32), oracle.shuffle(a, n)[0])
    ctx.close()


def test_suggest_schedule_is_reproducible(brr):
    from paper_2408_06213_gb300 import tune

    ctx = brr.Context(0)
    name, sched, times = tune.suggest_schedule(ctx, 100003, reps=2)
    assert name in times and times[name] == min(times.values())
    a = np.arange(100003, dtype=np.uint32)
    d = torch.from_numpy(a).cuda()
    ctx.shuffle(d, 5, sched=sched)
    ctx.check()
    z, _ = oracle.shuffle(a, 5, tuple(int(x) for x in sched.n_k), int(sched.k_max))
    assert np.array_equal(d.cpu().numpy().view(np.uint32), z)
    ctx.close()


def test_calibrated_cost_model_schedule(brr):
    """The Section 6.1 cost model with this GPU's measured costs gives a
    valid schedule, and shuffles under it equal the oracle's."""
    import math

    from paper_2408_06213_gb300 import tune

    ctx = brr.Context(0)
    costs = tune.gpu_costs(ctx)
    for v in costs["ns"].values():
        assert math.isfinite(v) and v > 0
    assert costs["c_rng"] > 0 and costs["c_div"] > 0
    nks, sched = tune.model_schedule(costs["c_rng"], costs["c_div"], k_max=6)
    assert all(nks[k] > nks[k + 1] for k in nks if k + 1 in nks)
    for n in (1000, 70001):
        a = np.arange(n, dtype=np.uint32)
        d = torch.from_numpy(a).cuda()
        ctx.shuffle(d, 3, sched=sched)
        ctx.check()
        z, _ = oracle.shuffle(a, 3, tuple(int(x) for x in sched.n_k), int(sched.k_max))
        assert np.array_equal(d.cpu().numpy().view(np.uint32), z)
    ctx.close()


def test_tune_fixed_then_dice(brr):
    # the fixed-bound kernel choice changes speed only: rolls after tuning
    # equal the oracle's
    from paper_2408_06213_gb300 import tune

    ctx = brr.Context(0)
    res = tune.tune_fixed(ctx, bounds=((6, 6), ((1 << 31) + 1, 2)), n_rolls=1 << 22, reps=2)
    assert res.settings["fixed_sweep"] in (0, 1) and len(res.trials) == 2
    assert tune.current(ctx)["fixed_sweep"] == res.settings["fixed_sweep"]
    for b, k in ((6, 6), ((1 << 31) + 1, 2), (1000, 6)):
        out = ctx.dice_fixed(b, k, 100003, 9)
        ctx.check()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.dice_fixed(b, k, 100003, 9))
    ctx.close()


def test_suggest_schedule_batched_is_reproducible(brr):
    """The schedule suggested for a batched layout (the 65,536-array
    configuration's distribution, fewer arrays) replays bit-exactly in the
    oracle with that schedule."""
    from paper_2408_06213_gb300 import inputs, tune

    ctx = brr.Context(0)
    data, offsets, seeds, max_len = inputs.batched_shuffles(1500, seed=21)
    cands = tune.schedule_candidates()
    cands.update(tune.model_candidates(ctx))
    name, sched, times = tune.suggest_schedule_batched(ctx, offsets, seeds, max_len, reps=1, candidates=cands)
    assert name in times and times[name] == min(times.values())
    d = torch.from_numpy(data).cuda()
    ctx.shuffle_batched(d, torch.from_numpy(offsets).cuda(), torch.from_numpy(seeds).cuda(), max_len, sched=sched)
    ctx.check()
    ref = oracle.shuffle_batched(data, offsets, seeds, tuple(int(x) for x in sched.n_k), int(sched.k_max))
    assert np.array_equal(d.cpu().numpy().view(np.uint32), ref)
    ctx.close()


def test_tune_batched_cached_second_call_times_nothing(brr, tmp_path):
    # the second call on the same layout applies the stored settings
    from paper_2408_06213_gb300 import inputs, tune

    ctx = brr.Context(0)
    _, offsets, _, max_len = inputs.batched_shuffles(n_arrays=512)
    path = str(tmp_path / "tune.json")
    first = tune.tune_batched_cached(ctx, offsets, max_len, path, reps=1, passes=1)
    assert first.trials
    ctx.tune(ctx.TUNE_SMALL_MAX, 0)
    second = tune.tune_batched_cached(ctx, offsets, max_len, path, reps=1, passes=1)
    assert not second.trials and second.settings == first.settings
    assert tune.current(ctx)["small_max"] == first.settings["small_max"]
    ctx.close()
