"""Seeded synthetic inputs for the batched-dice and shuffle workloads.

The same generators feed the GPU library and the CPU oracle in the tests and
the benchmark.  They hold none of the method's arithmetic: randomness comes
from numpy's PCG64 bit generator (a different generator from the SplitMix64
word stream the method consumes), and the only batching logic is the
left-to-right grouping of bounds under the product condition of Theorem 1.

Recipes (the paper's own experiments shuffle synthetic arrays, Section 7):
  dice    bounds b log-uniform on [2, 2^32]: u uniform in [0, 1) from 53 bits
          (chunk c of 2^24 rolls from PCG64(seed) jumped c times),
          b = clamp(floor(2^(1 + 31 u)), 2, 2^32); grouped greedily into
          batches of at most 6 bounds with product <= 2^64.  Fixed-bound runs
          use b in {6, 52, 1000, 2^31 + 1} in batches of the largest k <= 6
          with b^k <= 2^64.
  shuffle A[i] = i (uint32, n = 65,536, seed 42); random uint64 values
          (n = 2^24, seed 3).
  batched 65,536 arrays, sizes floor(16 * 4096^u) (log-uniform on
          [16, 65,536]), random uint32 values, per-array random seeds.
  serving Poisson arrivals at 20,000 requests/s; half full shuffles of
          n = floor(10^(2 + 5u)) uint32 elements (log-uniform 1e2..1e7), half
          samples of m = max(1, floor(10^(4u))) (log-uniform 1..1e4, at most
          n) from n drawn the same way; per-request random seeds.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
FIXED_BOUNDS = (6, 52, 1000, (1 << 31) + 1)
_grp = None


def _group_lib():
    global _grp
    if _grp is None:
        from . import build as _b

        path = _b.build_inputs_helper()
        lib = C.CDLL(path)
        lib.brr_inputs_group.restype = C.c_uint64
        lib.brr_inputs_group.argtypes = [C.c_void_p, C.c_uint64, C.c_uint32, C.c_void_p]
        _grp = lib
    return _grp


def _uniform53(gen: np.random.Generator, n: int) -> np.ndarray:
    raw = gen.bit_generator.random_raw(n)
    return (raw >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def dice_bounds(n: int, seed: int = 7, chunk: int = 1 << 24) -> np.ndarray:
    """Per-roll bounds as bm1 = b - 1 (uint32), b log-uniform on [2, 2^32].

    Chunk c of `chunk` rolls draws from PCG64(seed) jumped c times, so the
    result does not depend on how many threads fill it."""
    out = np.empty(n, dtype=np.uint32)

    def fill(c):
        s = c * chunk
        e = min(n, s + chunk)
        gen = np.random.Generator(np.random.PCG64(seed).jumped(c))
        u = _uniform53(gen, e - s)
        b = np.floor(np.exp2(1.0 + 31.0 * u))
        np.clip(b, 2.0, 4294967296.0, out=b)
        b -= 1.0
        out[s:e] = b.astype(np.uint32)

    n_chunks = (n + chunk - 1) // chunk
    if n_chunks <= 1:
        for c in range(n_chunks):
            fill(c)
    else:
        with cf.ThreadPoolExecutor(max_workers=min(n_chunks, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, range(n_chunks)))
    return out


def group_batches(bm1: np.ndarray, k_max: int = 6) -> np.ndarray:
    """CSR batch offsets (uint32): greedy, at most k_max bounds, product <= 2^64."""
    bm1 = np.ascontiguousarray(bm1, dtype=np.uint32)
    off = np.empty(bm1.size + 1, dtype=np.uint32)
    nb = _group_lib().brr_inputs_group(bm1.ctypes.data, bm1.size, k_max, off.ctypes.data)
    return off[: nb + 1].copy()


def dice_workload(n: int, seed: int = 7):
    bm1 = dice_bounds(n, seed)
    return bm1, group_batches(bm1)


def fixed_k(b: int, k_cap: int = 6) -> int:
    """Largest k <= k_cap with b^k <= 2^64."""
    k = 1
    while k < k_cap and b ** (k + 1) <= 1 << 64:
        k += 1
    return k


def shuffle_small(n: int = 65536):
    """A[i] = i, uint32; seed 42."""
    return np.arange(n, dtype=np.uint32), 42


def shuffle_large(n: int = 1 << 24, seed: int = 3):
    """Random uint64 values; shuffle seed 3."""
    gen = np.random.Generator(np.random.PCG64(seed))
    return gen.bit_generator.random_raw(n).astype(np.uint64), seed


def batched_shuffles(n_arrays: int = 65536, seed: int = 4, lo: int = 16, hi: int = 65536):
    """Returns (data uint32, offsets uint64 [n_arrays+1], seeds uint64, max_len)."""
    gen = np.random.Generator(np.random.PCG64(seed))
    u = _uniform53(gen, n_arrays)
    sizes = np.floor(lo * (hi / lo) ** u).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    offsets = np.zeros(n_arrays + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    data = gen.bit_generator.random_raw(total).astype(np.uint32)
    seeds = gen.bit_generator.random_raw(n_arrays).astype(np.uint64)
    return data, offsets, seeds, int(sizes.max()) if n_arrays else 0


def serving_trace(n_requests: int, rate: float = 20000.0, seed: int = 5,
                  n_lo: float = 1e2, n_hi: float = 1e7, m_hi: float = 1e4):
    """Poisson request stream: arrays of arrival time (s), kind (0 shuffle,
    1 sample), n, m (0 for shuffles) and seed."""
    gen = np.random.Generator(np.random.PCG64(seed))
    gaps = gen.exponential(1.0 / rate, size=n_requests)
    t = np.cumsum(gaps)
    kind = (gen.bit_generator.random_raw(n_requests) & np.uint64(1)).astype(np.int8)
    un = _uniform53(gen, n_requests)
    n = np.floor(n_lo * (n_hi / n_lo) ** un).astype(np.int64)
    um = _uniform53(gen, n_requests)
    m = np.maximum(1, np.floor(m_hi ** um)).astype(np.int64)
    m = np.minimum(m, n)
    m[kind == 0] = 0
    seeds = gen.bit_generator.random_raw(n_requests).astype(np.uint64)
    return t, kind, n, m, seeds
