"""Autotuner for the GPU shuffles and bulk dice.

Two kinds of choice are tuned here:

* **Kernel routing** (``brr_tune``): size-class limits of the batched CTA
  kernels and whether some classes use windowed reservations instead of
  chain resolution, the longest single array run in one CTA instead of the grid-wide
  passes, whether those passes run as one cooperative launch, and the
  fixed-bound dice kernel (sweep or tiled).  Every setting gives the same
  output, so the tuner applies the fastest one to the context.  It times a copy of the caller's layout (array lengths, element
  size) with CUDA events; the caller's own data is never touched.
* **Batch-size schedule** (Section 6, Table 2): the thresholds that pick k.
  The schedule decides which words each die uses, so a different schedule
  gives a different (equally uniform) permutation.  ``suggest_schedule``
  therefore only returns the fastest candidate; the caller decides whether
  to use it and must keep it with the results to reproduce them.  Besides
  fixed candidates it can try the schedule the Section 6.1 cost model gives
  with this GPU's measured costs (``gpu_costs``, ``model_schedule``).

The searches take a ``timer(settings) -> milliseconds`` callable, so the
search logic runs without a GPU (the tests drive it with synthetic costs).
Tuned routing settings can be kept in a JSON file keyed by GPU model and
layout (``tune_batched_cached``, ``cache_load``, ``cache_store``), so that a
layout seen before is set up without timing it again.
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


# ------------------------------------------------------------- tuning cache --
def layout_key(offsets, elem_bytes: int) -> str:
    """A key for a batched layout: the number of arrays, the element size
    and a hash of the array lengths (not of the data), so that a layout seen
    before is recognised whatever its contents."""
    import hashlib

    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    lengths = np.diff(off.astype(np.int64)) if off.size > 1 else np.zeros(0, dtype=np.int64)
    h = hashlib.sha256(np.ascontiguousarray(lengths, dtype=np.int64).tobytes()).hexdigest()[:16]
    return f"batched:{lengths.size}:{elem_bytes}:{h}"


def cache_load(path: str, device: str, key: str) -> dict | None:
    """Routing settings stored for (device, key) in the JSON cache at `path`,
    or None when the file, the device or the key is missing."""
    import json
    import os

    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None
    entry = data.get(device, {}).get(key)
    return dict(entry["settings"]) if entry and "settings" in entry else None


def cache_store(path: str, device: str, key: str, res: Result):
    """Record a tuning result for (device, key) in the JSON cache at `path`
    (other entries are kept; the file is replaced atomically)."""
    import json
    import os

    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    data.setdefault(device, {})[key] = {"settings": {k: int(v) for k, v in res.settings.items()}, "ms": res.ms}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


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


_PARAMS = {"small_max": 2, "medium_max": 3, "single_cta_max": 1, "grid_cooperative": 4, "fixed_sweep": 5,
           "ordered_push": 6, "window_route": 7}


def apply(ctx, settings: dict):
    """Set routing parameters on a context (names as in the Result)."""
    for name, value in settings.items():
        ctx.tune(_PARAMS[name], int(value))


def current(ctx) -> dict:
    return {name: ctx.tune_get(p) for name, p in _PARAMS.items()}


def tune_batched_cached(ctx, offsets, max_len: int, cache: str, elem_bytes: int = 4, **kw) -> Result:
    """tune_batched with a cache file: settings stored for this GPU model and
    layout are applied without timing anything (Result.trials empty);
    otherwise the layout is tuned and the result stored."""
    import torch

    if isinstance(offsets, torch.Tensor):
        offsets = offsets.cpu().view(torch.int64).numpy().view(np.uint64)
    device = torch.cuda.get_device_name(ctx.device)
    key = layout_key(offsets, elem_bytes)
    hit = cache_load(cache, device, key)
    if hit is not None:
        apply(ctx, hit)
        return Result(hit, float("nan"), [])
    res = tune_batched(ctx, offsets, max_len, elem_bytes, **kw)
    cache_store(cache, device, key, res)
    return res


def tune_batched(ctx, offsets, max_len: int, elem_bytes: int = 4, reps: int = 3, seed: int = 1,
                 passes: int = 2) -> Result:
    """Tune the size classes of brr_shuffle_batched, whether its chain
    kernels roll in barrier-separated rounds and whether the small and staged
    large arrays go to the windowed reservations, for arrays laid out by
    `offsets` (host or device, n_arrays + 1 element offsets), and apply the
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

    start = {k: v for k, v in current(ctx).items()
             if k in ("small_max", "medium_max", "ordered_push", "window_route")}
    res = coordinate_descent(start, {"small_max": SMALL_MAX, "medium_max": MEDIUM_MAX, "ordered_push": (0, 1),
                                     "window_route": (1, 0)}, timer, passes)
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


def tune_fixed(ctx, bounds=((6, 6), (52, 6), (1000, 6), ((1 << 31) + 1, 2)), n_rolls: int = 1 << 26,
               reps: int = 5) -> Result:
    """Choose the fixed-bound dice kernel (brr_dice_fixed: the sweep kernel
    or the tiled one) by the total time of `n_rolls` rolls of each (b, k) in
    `bounds`, and apply it to `ctx`."""
    import torch

    out = torch.empty(n_rolls, dtype=torch.int32, device=ctx.device).view(torch.uint32) \
        if hasattr(torch, "uint32") else torch.empty(n_rolls, dtype=torch.int32, device=ctx.device)

    def timer(settings):
        apply(ctx, settings)
        return sum(_events_timer(lambda b=b, k=k: ctx.dice_fixed(b, k, n_rolls, 7, out=out), reps)
                   for b, k in bounds)

    res = coordinate_descent({"fixed_sweep": current(ctx)["fixed_sweep"]}, {"fixed_sweep": (0, 1)}, timer, 1)
    apply(ctx, res.settings)
    ctx.check()
    return res


# ------------------------------------------------------- cost model (6.1) --
def cost_avg(k: int, n, L: int = 64, c_rng: float = 2.0, c_div: float = 16.0):
    """Expected cost per die of batches of k at remaining length n (Section
    6.1), in multiplications: each attempt costs a word and k multiplies and
    is repeated 1/(1 - p2) times, where p2 = (2^L mod b) / 2^L; the first
    threshold fails with p1 = b / 2^L and then costs k-1 multiplies and a
    division; b = n (n-1) ... (n-k+1).  n may be a numpy array of uint64;
    lengths whose b exceeds 2^L get +inf."""
    n = np.atleast_1d(np.asarray(n, dtype=np.uint64))
    b = np.ones_like(n)
    ok = np.ones(n.shape, dtype=bool)
    limit = np.uint64((1 << L) - 1) if L < 64 else None
    with np.errstate(over="ignore"):
        for m in range(k):
            f = n - np.uint64(m)
            ok &= n > np.uint64(m)
            # b * f <= 2^L (b == 2^L only when the product is exactly 2^L: L < 64)
            hi = np.where(f > 0, np.uint64(0xFFFFFFFFFFFFFFFF) // np.maximum(f, np.uint64(1)), np.uint64(0))
            ok &= b <= hi
            b = b * f
    if L < 64:
        ok &= b <= np.uint64(1 << L)
        rem = np.where(ok, np.uint64(1 << L) % np.maximum(b, np.uint64(1)), np.uint64(0))
        W = float(1 << L)
    else:
        ok &= b != 0
        rem = np.where(ok, (np.uint64(0) - b) % np.maximum(b, np.uint64(1)), np.uint64(0))
        W = 18446744073709551616.0
    p1 = b.astype(np.float64) / W
    p2 = rem.astype(np.float64) / W
    with np.errstate(divide="ignore", invalid="ignore"):
        c = ((c_rng + k) / (1.0 - p2) + (c_div + k - 1) * p1) / k
    return np.where(ok, c, np.inf)


def model_nk(k: int, L: int = 64, c_rng: float = 2.0, c_div: float = 16.0, n_limit: int = 1 << 33,
             chunk: int = 1 << 22) -> int:
    """n_k (Section 6.1): the largest n such that batches of k cost less per
    die than batches of k-1 for every length from k up to n (0 if past
    n_limit).  Scans upward in chunks."""
    if k < 2:
        return 0
    lo = max(k, _certain_prefix(k, L, c_rng, c_div, n_limit) + 1)
    while lo <= n_limit:
        hi = min(n_limit, lo + chunk - 1)
        n = np.arange(lo, hi + 1, dtype=np.uint64)
        worse = ~(cost_avg(k, n, L, c_rng, c_div) < cost_avg(k - 1, n, L, c_rng, c_div))
        if worse.any():
            return int(n[int(np.argmax(worse))]) - 1
        lo = hi + 1
    return 0


def _certain_prefix(k: int, L: int, c_rng: float, c_div: float, n_limit: int) -> int:
    """Largest n such that batches of k are certainly cheaper than k-1 for
    every length up to n, from bounds alone: p2 < p1 (2^L mod b < b) gives
    c_avg(k) <= ((c_rng + k)/(1 - p1) + (c_div + k - 1) p1) / k, and
    c_avg(k-1) >= (c_rng + k - 1)/(k - 1); the upper bound grows with n.
    The exact scan can start after it (0: no such n)."""
    W = float(1 << L)
    low = (c_rng + k - 1) / (k - 1) * (1.0 - 1e-12)

    def holds(n):
        b = 1
        for m in range(k):
            b *= n - m
        p1 = b / W
        if p1 >= 1.0:
            return False
        return ((c_rng + k) / (1.0 - p1) + (c_div + k - 1) * p1) / k < low

    lo, hi = k - 1, n_limit  # holds(lo) is taken as true, hi is a bound to search under
    if not holds(k):
        return 0
    lo = k
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if holds(mid):
            lo = mid
        else:
            hi = mid
    return lo - 1  # one below, against rounding at the edge


def gpu_costs(ctx, large_products: bool = True) -> dict:
    """c_rng and c_div of the cost model measured on this GPU (brr_calibrate),
    in units of one chain step.  The threshold of products at or above 2^48
    (the shuffles' batches) or below 2^40 stands for the division."""
    ns = ctx.calibrate()
    thr = ns["threshold_large"] if large_products else ns["threshold_small"]
    return {"c_rng": ns["word"] / ns["step"], "c_div": thr / ns["step"], "ns": ns}


def model_schedule(c_rng: float, c_div: float, k_max: int = 6, L: int = 64, round_pow2: bool = True):
    """A schedule from the cost model: n_k for k = 2..k_max, each rounded
    down to a power of two as Section 7 does with Table 2 (round_pow2).
    Returns (n_k dict, Schedule)."""
    from . import schedule

    nks = {}
    for k in range(2, k_max + 1):
        v = model_nk(k, L, c_rng, c_div)
        if v <= 0:
            break
        nks[k] = 1 << (v.bit_length() - 1) if round_pow2 else v
    return nks, schedule(n_k=nks) if nks else schedule(k_max=1)


def schedule_candidates():
    """Batch-size schedules to compare: the paper's (Table 2 rounded down to
    powers of two) with k capped at 1..6, and Table 2's L = 64 column as
    printed."""
    from . import schedule

    cands = {f"paper_kmax{k}": schedule(k_max=k) for k in range(1, 7)}
    cands["table2_L64"] = schedule(n_k={2: 1358187913, 3: 929104, 4: 26573, 5: 3225, 6: 815})
    return cands


def model_candidates(ctx, k_max: int = 6) -> dict:
    """The cost-model schedule with this GPU's measured costs (rounded down
    to powers of two, and as computed), as candidates for suggest_schedule."""
    c = gpu_costs(ctx)
    out = {}
    for pow2 in (True, False):
        nks, sc = model_schedule(c["c_rng"], c["c_div"], k_max=k_max, round_pow2=pow2)
        out["gpu_model" + ("_pow2" if pow2 else "")] = sc
    return out


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


def suggest_schedule_batched(ctx, offsets, seeds, max_len: int, elem_bytes: int = 4, reps: int = 3,
                             candidates: dict | None = None):
    """Time brr_shuffle_batched over the caller's layout (`offsets` and
    `seeds`, host arrays) under each candidate schedule and return (name,
    schedule, {name: ms}).  Nothing is applied: the schedule decides which
    words every die uses, so a caller that adopts it must keep it with the
    results (the oracle replays a shuffle under any valid schedule)."""
    import torch

    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    dev = ctx.device
    dtype = torch.int32 if elem_bytes == 4 else torch.int64
    data = torch.zeros(max(int(off[-1]), 1), dtype=dtype, device=dev)  # values do not affect timing
    o = torch.from_numpy(off).to(dev)
    sd = torch.from_numpy(np.ascontiguousarray(seeds, dtype=np.uint64)).to(dev)
    cands = candidates or schedule_candidates()
    times = {name: _events_timer(lambda sc=sc: ctx.shuffle_batched(data, o, sd, max_len, sched=sc), reps)
             for name, sc in cands.items()}
    ctx.check()
    best = min(times, key=times.get)
    return best, cands[best], times
