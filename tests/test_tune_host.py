"""Host logic of the autotuner (no GPU): the searches driven by synthetic
cost functions with known optima."""
from paper_2408_06213_gb300 import tune


def test_coordinate_descent_finds_separable_optimum():
    space = {"a": (0, 1, 2, 3, 4), "b": (10, 20, 30)}
    cost = lambda s: (s["a"] - 3) ** 2 + abs(s["b"] - 20) + 1.0
    res = tune.coordinate_descent({"a": 0, "b": 10}, space, cost)
    assert res.settings == {"a": 3, "b": 20}
    assert res.ms == 1.0
    # every setting is timed at most once
    keys = [tuple(sorted(s.items())) for s, _ in res.trials]
    assert len(keys) == len(set(keys))


def test_coordinate_descent_keeps_start_when_it_is_best():
    res = tune.coordinate_descent({"a": 1}, {"a": (0, 1, 2)}, lambda s: abs(s["a"] - 1))
    assert res.settings == {"a": 1} and res.ms == 0


def test_coordinate_descent_second_pass_uses_interaction():
    # the best b depends on a: a second sweep is needed to reach (2, 2)
    cost = lambda s: 10 - (3 if s["a"] == 2 else 0) - (4 if (s["a"] == 2 and s["b"] == 2) else 0) \
        - (1 if s["b"] == 1 else 0)
    res = tune.coordinate_descent({"a": 0, "b": 0}, {"a": (0, 1, 2), "b": (0, 1, 2)}, cost, passes=3)
    assert res.settings == {"a": 2, "b": 2}


def test_crossover_takes_the_prefix_where_cta_wins():
    cta = {1: 1, 2: 2, 4: 5, 8: 4}
    grid = {1: 3, 2: 3, 4: 3, 8: 9}
    assert tune.crossover([1, 2, 4, 8], cta.get, grid.get) == 2  # stops at the first loss
    assert tune.crossover([1, 2], lambda n: 9, lambda n: 1) == 0


def test_cost_model_reproduces_table2():
    # Section 6.1 with c_rng = 2, c_div = 16 gives Table 2 (golden file),
    # all ten entries
    import os

    gold = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_estimated_nk.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        L, k, n = (int(x) for x in line.split())
        gold[(L, k)] = n
    assert len(gold) == 10, "golden file not parsed"
    for (L, k), n in gold.items():
        assert tune.model_nk(k, L) == n, (L, k)


def test_cost_model_matches_the_oracle_for_other_costs():
    import oracle

    for c_rng, c_div in ((4.0, 8.0), (1.0, 30.0), (9.5, 3.0)):
        for k in (4, 5, 6):
            assert tune.model_nk(k, 64, c_rng, c_div) == oracle.nk(k, 64, c_rng, c_div), (c_rng, c_div, k)
        for k in (2, 3):
            assert tune.model_nk(k, 32, c_rng, c_div) == oracle.nk(k, 32, c_rng, c_div), (c_rng, c_div, k)


def test_cost_avg_is_inf_past_the_word():
    import numpy as np

    c = tune.cost_avg(3, np.array([5, 2_600_000, 2_700_000], dtype=np.uint64))
    assert np.isfinite(c[0]) and np.isfinite(c[1]) and np.isinf(c[2])  # 2.7e6^3 > 2^64 > 2.6e6^3


def test_tuning_cache_round_trip(tmp_path):
    import numpy as np

    path = str(tmp_path / "tune.json")
    off = np.array([0, 5, 9, 100], dtype=np.uint64)
    key = tune.layout_key(off, 4)
    # the key depends on the lengths and element size, not on where the arrays start
    assert key == tune.layout_key(off + np.uint64(7), 4)
    assert key != tune.layout_key(off, 8)
    assert key != tune.layout_key(np.array([0, 5, 10, 100], dtype=np.uint64), 4)
    assert tune.cache_load(path, "GPU A", key) is None
    res = tune.Result({"small_max": 1024, "medium_max": 8192}, 1.5, [])
    tune.cache_store(path, "GPU A", key, res)
    tune.cache_store(path, "GPU B", key, tune.Result({"small_max": 2048}, 2.0, []))
    assert tune.cache_load(path, "GPU A", key) == {"small_max": 1024, "medium_max": 8192}
    assert tune.cache_load(path, "GPU B", key) == {"small_max": 2048}
    assert tune.cache_load(path, "GPU A", "other") is None
    # a damaged file reads as empty and is replaced by the next store
    with open(path, "w") as f:
        f.write("{not json")
    assert tune.cache_load(path, "GPU A", key) is None
    tune.cache_store(path, "GPU A", key, res)
    assert tune.cache_load(path, "GPU A", key) == {"small_max": 1024, "medium_max": 8192}
