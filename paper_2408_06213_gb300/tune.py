"""Autotuner for the GPU shuffles.

Two kinds of choice are tuned here:

* **Kernel routing** (``brr_tune``): size-class limits of the batched CTA
  kernels, the longest single array run in one CTA instead of the grid-wide
  passes, and whether those passes run as one cooperative launch.  Every
  setting gives the same output, so the tuner applies the fastest one to the
  context.  It times a copy of the caller's layout (array lengths, element
  size) with CUDA events; the caller's own data is never touched.
* **Batch-size schedule** (Section 6, Table 2): the thresholds that pick k.
  The schedule decides which words each die uses, so a different schedule
  gives a different (equally uniform) permutation.  ``suggest_schedule``
  therefore only returns the fastest candidate; the caller decides whether
  to use it and must keep it with the results to reproduce them.

The searches take a ``timer(settings) -> milliseconds`` callable, so the
search logic runs without a GPU (the tests drive it with synthetic costs).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Iterable

import numpy as np

# candidate values of each routing parameter, in the order tried
SMALL_MAX = (0, 256, 512, 1024, 2048, 4096)
MEDIUM_MAX = (0, 2048, 4096, 8192, 16384, 28672)
SINGLE_SIZES = (1024, 2048, 4096, 8192, 16384, 32768, 65536)


@dataclasses.dataclass
class Result:
    settings: dict
    ms: float
    trials: list  # (settings, ms) in the order measured


def coordinate_descent(start: dict, space: dict[str, Iterable], timer: Callable[[dict], float],
                       passes: int = 2) -> Result:
    """Minimise timer() one parameter at a time over `space` (each value
    timed with the others held), `passes` sweeps, starting from `start`.
    Settings already measured are not timed again."""
    best = dict(start)
    seen: dict[tuple, float] = {}
    trials = []

    def cost(s):
        key = tuple(sorted(s.items()))
        if key not in seen:
            seen[key] = float(timer(dict(s)))
            trials.append((dict(s), seen[key]))
        return seen[key]

    best_ms = cost(best)
    for _ in range(passes):
        changed = False
        for name, values in space.items():
            for v in values:
                if v == best[name]:
                    continue
                cand = dict(best)
                cand[name] = v
                ms = cost(cand)
                if ms < best_ms:
                    best, best_ms, changed = cand, ms, True
        if not changed:
            break
    return Result(best, best_ms, trials)


def crossover(sizes: Iterable[int], cta_ms: Callable[[int], float], grid_ms: Callable[[int], float]) -> int:
    """Longest size of the increasing prefix of `sizes` on which one CTA is
    at least as fast as the grid passes (0 if it never is)."""
    best = 0
    for n in sizes:
        if cta_ms(n) <= grid_ms(n):
            best = n
        else:
            break
    return best


# ----------------------------------------------------------------- GPU side --
def _events_timer(fn, reps: int, stream=None) -> float:
    import torch

    stream = stream or torch.cuda.current_stream()
    fn()  # warm-up: kernel setup and scratch growth are not timed
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


_PARAMS = {"small_max": 2, "medium_max": 3, "single_cta_max": 1, "grid_cooperative": 4}


def apply(ctx, settings: dict):
    """Set routing parameters on a context (names as in the Result)."""
    for name, value in settings.items():
        ctx.tune(_PARAMS[name], int(value))


def current(ctx) -> dict:
    return {name: ctx.tune_get(p) for name, p in _PARAMS.items()}


def tune_batched(ctx, offsets, max_len: int, elem_bytes: int = 4, reps: int = 3, seed: int = 1,
                 passes: int = 2) -> Result:
    """Tune the size classes of brr_shuffle_batched for arrays laid out by
    `offsets` (host or device, n_arrays + 1 element offsets) and apply the
    fastest to `ctx`."""
    import torch

    if isinstance(offsets, torch.Tensor):
        offsets = offsets.cpu().view(torch.int64).numpy().view(np.uint64)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    n_arrays = off.size - 1
    dev = ctx.device
    dtype = torch.int32 if elem_bytes == 4 else torch.int64
    data = torch.zeros(max(int(off[-1]), 1), dtype=dtype, device=dev)  # values do not affect timing
    o = torch.from_numpy(off).to(dev)
    rng = np.random.default_rng(seed)
    s = torch.from_numpy(rng.integers(0, 1 << 63, size=n_arrays, dtype=np.uint64)).to(dev)

    def timer(settings):
        apply(ctx, settings)
        return _events_timer(lambda: ctx.shuffle_batched(data, o, s, max_len), reps)

    start = {k: v for k, v in current(ctx).items() if k in ("small_max", "medium_max")}
    res = coordinate_descent(start, {"small_max": SMALL_MAX, "medium_max": MEDIUM_MAX}, timer, passes)
    apply(ctx, res.settings)
    ctx.check()
    return res


def tune_single(ctx, elem_bytes: int = 4, sizes: Iterable[int] = SINGLE_SIZES, reps: int = 5,
                large: int = 1 << 22) -> Result:
    """Tune brr_shuffle of one array: the longest length run in one CTA, and
    cooperative or per-pass grid launches (timed at 65,536 and `large`
    elements); applies the result to `ctx`."""
    import torch

    sizes = sorted(set(int(n) for n in sizes))
    dtype = torch.int32 if elem_bytes == 4 else torch.int64
    bufs = {n: torch.zeros(n, dtype=dtype, device=ctx.device) for n in set(sizes) | {65536, large}}
    trials = []

    def ms_for(n, cta_max, coop):
        apply(ctx, {"single_cta_max": cta_max, "grid_cooperative": coop})
        t = _events_timer(lambda: ctx.shuffle(bufs[n], 7), reps)
        trials.append(({"n": n, "single_cta_max": cta_max, "grid_cooperative": coop}, t))
        return t

    coop_ms = {c: ms_for(65536, 0, c) + ms_for(large, 0, c) for c in (0, 1)}
    coop = 1 if coop_ms[1] <= coop_ms[0] else 0
    cta_max = crossover(sizes, lambda n: ms_for(n, 65536, coop), lambda n: ms_for(n, 0, coop))
    settings = {"single_cta_max": cta_max, "grid_cooperative": coop}
    apply(ctx, settings)
    ctx.check()
    return Result(settings, min(coop_ms.values()), trials)


def schedule_candidates():
    """Batch-size schedules to compare: the paper's (Table 2 rounded down to
    powers of two) with k capped at 1..6, and Table 2's L = 64 column as
    printed."""
    from . import schedule

    cands = {f"paper_kmax{k}": schedule(k_max=k) for k in range(1, 7)}
    cands["table2_L64"] = schedule(n_k={2: 1358187913, 3: 929104, 4: 26573, 5: 3225, 6: 815})
    return cands


def suggest_schedule(ctx, n: int, elem_bytes: int = 4, reps: int = 5, candidates: dict | None = None):
    """Time brr_shuffle of n elements under each candidate schedule and
    return (name, schedule, {name: ms}).  Nothing is applied: the schedule
    is part of a shuffle's definition (see the module docstring)."""
    import torch

    dtype = torch.int32 if elem_bytes == 4 else torch.int64
    buf = torch.zeros(n, dtype=dtype, device=ctx.device)
    cands = candidates or schedule_candidates()
    times = {name: _events_timer(lambda sc=sc: ctx.shuffle(buf, 7, sched=sc), reps) for name, sc in cands.items()}
    ctx.check()
    best = min(times, key=times.get)
    return best, cands[best], times
