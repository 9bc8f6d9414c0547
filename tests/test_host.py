"""Host-side logic of libbrr (runs without a GPU): the C ABI loads and exports
every entry point include/brr.h declares, the batch planner matches the
oracle's sequential batch loop, and the seeded input generators behave as
documented."""
import math
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def brr():
    import __graft_entry__ as g

    g.build()
    import paper_2408_06213_gb300 as brr

    return brr


def _header_functions():
    text = open(os.path.join(ROOT, "include", "brr.h")).read()
    return sorted(set(re.findall(r"^\s*(?:brr_status|void|const char \*)\s*\*?\s*(brr_\w+)\s*\(", text, re.M)))


def test_abi_exports_every_declared_symbol(brr):
    import ctypes

    names = _header_functions()
    assert len(names) >= 14
    L = ctypes.CDLL(brr._lib.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name
    assert set(names) <= set(brr.exported_symbols()) | {"brr_shuffle_plan"}


def test_status_strings(brr):
    for s in range(7):
        assert brr.lib().brr_status_str(s).decode().startswith("BRR_")


def _oracle_batches(n, stop, nk, k_max):
    """The batch loop of the oracle's shuffle/sample, as (i, k) pairs."""
    out, i = [], n
    while i > stop:
        k = min(oracle.k_rule(i, nk, k_max), i - stop)
        out.append((i, k))
        i -= k
    return out


def _expand(segs):
    out = []
    for s in segs:
        for c in range(s["count"]):
            out.append((s["i0"] - c * s["k"], s["k"]))
    return out


SCHEDS = [
    (oracle.PAPER_NK, 6),
    (oracle.PAPER_NK, 1),
    (oracle.PAPER_NK, 2),
    (oracle.PAPER_NK, 4),
    ((0, 0, 1358187913, 929104, 26573, 3225, 815, 305, 146), 8),  # Table 2, L = 64
    ((0, 0, 50, 100, 20, 0, 0, 0, 0), 4),  # non-monotone thresholds
]


@pytest.mark.parametrize("nk,k_max", SCHEDS)
def test_plan_matches_oracle_loop(brr, nk, k_max):
    sched = brr.schedule({k: nk[k] for k in range(2, 9)}, k_max=k_max)
    ns = list(range(0, 40)) + [511, 512, 513, 514, 2047, 2048, 2049, 2050, 16383, 16384, 16385, 16386,
                               65535, 65536, 65537, 100003, (1 << 19) - 1, 1 << 19, (1 << 19) + 1, (1 << 19) + 2]
    for n in ns:
        for stop in sorted({1, max(n - 1, 1), max(n - 5, 1), max(n // 2, 1), max(n - 700, 1)}):
            if stop > max(n, 1):
                continue
            segs, nb = brr.plan(n, stop, sched)
            ref = _oracle_batches(n, stop, nk, k_max)
            assert _expand(segs) == ref, (n, stop)
            assert nb == len(ref)
            for s in segs:
                assert s["u"] == math.prod(range(s["i0"] - s["k"] + 1, s["i0"] + 1))


def test_plan_large_n_segment_count(brr):
    segs, nb = brr.plan((1 << 32) - 1)
    assert [s["k"] for s in segs][:6] == [1, 2, 3, 4, 5, 6]
    assert sum(s["count"] * s["k"] for s in segs) == (1 << 32) - 2


def test_plan_rejects_invalid(brr):
    from paper_2408_06213_gb300 import BrrError

    with pytest.raises(BrrError):
        brr.plan(1 << 32)
    with pytest.raises(BrrError):  # 2^40 * (2^40 - 1) > 2^64
        brr.plan(1000, 1, brr.schedule({2: 1 << 40}))
    with pytest.raises(BrrError):
        brr.plan(10, 11)


# --------------------------------------------------------------- inputs --
def test_dice_inputs_grouping():
    from paper_2408_06213_gb300 import inputs

    bm1, off = inputs.dice_workload(200000, seed=7)
    b = bm1.astype(object) + 1
    assert min(b) >= 2 and max(b) <= 1 << 32
    assert off[0] == 0 and off[-1] == bm1.size and np.all(np.diff(off.astype(np.int64)) >= 1)
    ks = np.diff(off.astype(np.int64))
    assert ks.max() <= 6 and ks[:-1].min() >= 2
    for g in range(0, len(off) - 1, 97):
        s, e = int(off[g]), int(off[g + 1])
        p = math.prod(b[s:e])
        assert p <= 1 << 64
        if e < bm1.size and e - s < 6:  # greedy: the next bound would not fit
            assert p * b[e] > 1 << 64
    # log-uniform: log2(b) roughly uniform on [1, 32]
    lg = np.log2(bm1.astype(np.float64) + 1)
    hist = np.histogram(lg, bins=31, range=(1, 32))[0]
    assert hist.min() > 0.8 * hist.mean() and hist.max() < 1.2 * hist.mean()
    bm1b, offb = inputs.dice_workload(200000, seed=7)
    assert np.array_equal(bm1, bm1b) and np.array_equal(off, offb)


def test_fixed_k():
    from paper_2408_06213_gb300 import inputs

    assert [inputs.fixed_k(b) for b in inputs.FIXED_BOUNDS] == [6, 6, 6, 2]


def test_batched_inputs():
    from paper_2408_06213_gb300 import inputs

    data, offsets, seeds, max_len = inputs.batched_shuffles(4096, seed=4)
    sizes = np.diff(offsets.astype(np.int64))
    assert sizes.min() >= 16 and sizes.max() <= 65536 and max_len == sizes.max()
    assert data.size == offsets[-1] and seeds.size == 4096
    # log-uniform: median near sqrt(16 * 65536) = 1024
    assert 700 < np.median(sizes) < 1500


def test_serving_trace():
    from paper_2408_06213_gb300 import inputs

    t, kind, n, m, seeds = inputs.serving_trace(20000)
    assert abs(t[-1] - 1.0) < 0.05  # 20k requests at 20k/s
    assert 0.45 < kind.mean() < 0.55
    assert n.min() >= 100 and n.max() <= 10 ** 7
    assert np.all(m[kind == 1] >= 1) and np.all(m <= n) and np.all(m[kind == 0] == 0)


def test_l32_schedule_matches_oracle(brr):
    # the library's L = 32 schedule is the oracle's (Table 2's L = 32 column
    # rounded down); its plan matches the oracle's batch loop
    s = brr.l32_schedule()
    assert s.k_max == oracle.L32_KMAX
    assert [int(s.n_k[k]) for k in range(9)] == list(oracle.L32_NK)
    for n in (2, 65, 513, 16385, 100000):
        segs, nb = brr.plan(n, 1, s)
        assert _expand(segs) == _oracle_batches(n, 1, oracle.L32_NK, oracle.L32_KMAX)
