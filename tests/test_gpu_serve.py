"""Serving (continuous batching): every request's result is bit-identical
whether it runs alone or mixed with overlapping waves, and matches the
oracle."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def engine_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_2408_06213_gb300 import serve

    return serve


def _trace(n_req, seed, n_hi=3e5):
    from paper_2408_06213_gb300 import inputs

    return inputs.serving_trace(n_req, rate=20000.0, seed=seed, n_hi=n_hi)


@pytest.mark.parametrize("realtime", [False, True])
def test_serving_mix_equals_alone(engine_mod, realtime):
    serve = engine_mod
    t, kind, n, m, seeds = _trace(600, seed=7)
    eng = serve.ServeEngine(0, n_slots=3, hbm_budget=64 << 20, max_wave=64, max_n=int(n.max()),
                            max_m=int(m.max()))
    stats = eng.run_trace(t, kind, n, m, seeds, realtime=realtime)
    reqs = stats["requests_list"]
    assert stats["requests"] == 600 and stats["p99_ms"] >= stats["p50_ms"] > 0
    import paper_2408_06213_gb300 as brr

    ctx = brr.Context(0)
    rng = np.random.default_rng(1)
    for r in reqs:
        got = r.result.cpu().numpy().view(np.uint32)
        if r.kind == serve.SHUFFLE:
            alone = torch.arange(r.n, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
            ctx.shuffle(alone, r.seed)
        else:
            alone = ctx.sample(r.n, r.m, r.seed)
        ctx.check()
        assert np.array_equal(got, alone.cpu().numpy().view(np.uint32)), r.rid
    for r in rng.choice(reqs, 40, replace=False):
        got = r.result.cpu().numpy().view(np.uint32)
        if r.kind == serve.SHUFFLE:
            ref = oracle.shuffle(np.arange(r.n, dtype=np.uint32), r.seed)[0]
        else:
            ref = oracle.sample(r.n, r.m, r.seed)
        assert np.array_equal(got, ref), r.rid
    ctx.close()


def test_serving_assigned_seeds_distinct(engine_mod):
    serve = engine_mod
    eng = serve.ServeEngine(0, n_slots=2, hbm_budget=16 << 20, max_wave=8)
    t = np.linspace(0, 0.001, 64)
    kind = np.ones(64, dtype=np.int8)
    n = np.full(64, 1000)
    m = np.full(64, 10)
    stats = eng.run_trace(t, kind, n, m, None, realtime=False)
    outs = {tuple(r.result.cpu().numpy().tolist()) for r in stats["requests_list"]}
    assert len(outs) == 64  # every request without a seed got its own


def test_serving_waves_overlap_on_the_device(engine_mod):
    """Requests large enough that a wave's device time exceeds the host's
    launch time, all arriving at once: the waves of different slots run on
    the device at the same time (their start-to-end event intervals
    overlap), and every result still equals the request run alone."""
    serve = engine_mod
    t, kind, n, m, seeds = _trace(120, seed=11, n_hi=1e7)
    eng = serve.ServeEngine(0, n_slots=4, hbm_budget=1 << 30, max_wave=8, max_n=int(n.max()),
                            max_m=int(m.max()))
    stats = eng.run_trace(t, kind, n, m, seeds, realtime=False)
    assert stats["waves"] >= 4
    assert stats["device_max_concurrent_waves"] >= 2, stats["device_max_concurrent_waves"]
    import paper_2408_06213_gb300 as brr

    ctx = brr.Context(0)
    for r in stats["requests_list"]:
        got = r.result.cpu().numpy().view(np.uint32)
        if r.kind == serve.SHUFFLE:
            alone = torch.arange(r.n, dtype=torch.int32, device="cuda").view(torch.uint32)
            ctx.shuffle(alone, r.seed)
        else:
            alone = ctx.sample(r.n, r.m, r.seed)
        ctx.check()
        assert np.array_equal(got, alone.cpu().numpy().view(np.uint32)), r.rid
    ctx.close()
