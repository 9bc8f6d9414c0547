"""CPU oracle for batched ranged random integers (arXiv 2408.06213).

TEST INFRASTRUCTURE ONLY.  This package wraps ``brr_oracle.c``, a plain,
sequential C implementation of the paper's algorithms (Theorem 1, Algorithms
1-4, the Section 6.1 cost model).  It shares no code with the GPU library:
only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import it.

Every function takes and returns numpy arrays; the shared library is compiled
with the system C compiler on first use (or by ``build()``).
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ERETRY = 0, 1, 4

# Schedule used in the paper's experiments (Section 7): batches of 2 up to
# 2^30 remaining elements, 3 up to 2^19, 4 up to 2^14, 5 up to 2^11 and 6 up
# to 2^9 -- Table 2's L = 64 estimates rounded down to powers of two.
PAPER_NK = (0, 0, 1 << 30, 1 << 19, 1 << 14, 1 << 11, 1 << 9, 0, 0)
PAPER_KMAX = 6


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        ):
            os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.run(
                ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                check=True,
            )
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB_PATH)
    u64, u32, i32, vp = C.c_uint64, C.c_uint32, C.c_int, C.c_void_p
    sig = {
        "orc_mix64": (u64, [u64]),
        "orc_word": (u64, [u64, u64, u64]),
        "orc_chain": (u64, [C.c_uint, vp, C.c_uint, u64, vp]),
        "orc_threshold": (i32, [C.c_uint, vp, C.c_uint, vp]),
        "orc_lemire": (i32, [u64, u64, u64, vp]),
        "orc_roll_batch": (i32, [vp, C.c_uint, u64, u64, vp, vp]),
        "orc_dice": (i32, [vp, vp, u64, u64, u64, vp]),
        "orc_dice_fixed": (i32, [u64, C.c_uint, u64, u64, vp]),
        "orc_dice_range": (i32, [vp, vp, u64, u64, u64, vp]),
        "orc_dice_fixed_range": (i32, [u64, C.c_uint, u64, u64, u64, u64, vp]),
        "orc_k_rule": (C.c_uint, [u64, vp, C.c_uint]),
        "orc_shuffle": (i32, [vp, u64, u32, u64, vp, C.c_uint, vp]),
        "orc_apply_swaps": (i32, [vp, u64, u32, vp]),
        "orc_shuffle_batched": (i32, [vp, vp, u64, u32, vp, vp, C.c_uint]),
        "orc_sample": (i32, [u64, u64, u64, vp, C.c_uint, vp]),
        "orc_partial_shuffle_word_L": (i32, [C.c_uint, vp, u64, C.c_uint, u64, u64, vp]),
        "orc_cost_avg": (C.c_double, [C.c_uint, u64, C.c_uint, C.c_double, C.c_double]),
        "orc_naive_shuffle": (C.c_int, [vp, u64, C.c_uint32, u64, vp, C.c_uint, vp]),
        "orc_naive_digits": (None, [u64, u64, C.c_uint, vp]),
        "orc_nk": (u64, [C.c_uint, C.c_uint, C.c_double, C.c_double, u64]),
        "orc_chacha_block": (None, [vp, C.c_uint, vp]),
        "orc_chacha_input": (None, [u64, u64, vp]),
        "orc_src_bits": (C.c_uint, [C.c_uint]),
        "orc_word_src": (u64, [C.c_uint, u64, u64, u64]),
        "orc_roll_batch_src": (i32, [C.c_uint, vp, C.c_uint, u64, u64, vp, vp]),
        "orc_shuffle_src": (i32, [C.c_uint, vp, u64, u32, u64, vp, C.c_uint, vp]),
        "orc_dice_fixed_src": (i32, [C.c_uint, u64, C.c_uint, u64, u64, vp]),
        "orc_dice_src": (i32, [C.c_uint, vp, vp, u64, u64, u64, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _check(st: int, what: str):
    if st != OK:
        raise OracleError(f"{what}: oracle status {st}")


def _nk_array(nk) -> np.ndarray:
    a = np.zeros(9, dtype=np.uint64)
    nk = list(nk)
    a[: len(nk)] = nk
    return a


# ------------------------------------------------------------------ words --
def mix64(z: int) -> int:
    return _load().orc_mix64(z)


def word(seed: int, g: int, a: int) -> int:
    return _load().orc_word(seed, g, a)


# ------------------------------------------------------- Theorem 1 chain --
def chain(L: int, b, r0: int):
    """Return (digits a_1..a_k, r_k) of the Theorem 1 chain at word size L."""
    b = np.ascontiguousarray(b, dtype=np.uint64)
    a = np.zeros(len(b), dtype=np.uint64)
    rk = _load().orc_chain(L, _ptr(b), len(b), r0, _ptr(a))
    return [int(x) for x in a], int(rk)


def threshold(L: int, b) -> int:
    b = np.ascontiguousarray(b, dtype=np.uint64)
    t = np.zeros(1, dtype=np.uint64)
    _check(_load().orc_threshold(L, _ptr(b), len(b), _ptr(t)), "threshold")
    return int(t[0])


def lemire(b: int, seed: int, g: int) -> int:
    out = np.zeros(1, dtype=np.uint64)
    _check(_load().orc_lemire(b, seed, g, _ptr(out)), "lemire")
    return int(out[0])


def roll_batch(b, seed: int, g: int):
    """Algorithm 3 on the words of batch g: returns (digits, attempts used)."""
    b = np.ascontiguousarray(b, dtype=np.uint64)
    a = np.zeros(len(b), dtype=np.uint64)
    att = np.zeros(1, dtype=np.uint32)
    _check(_load().orc_roll_batch(_ptr(b), len(b), seed, g, _ptr(a), _ptr(att)), "roll_batch")
    return [int(x) for x in a], int(att[0])


# ------------------------------------------------------------------- dice --
def dice(bm1: np.ndarray, off: np.ndarray | None, seed: int) -> np.ndarray:
    bm1 = np.ascontiguousarray(bm1, dtype=np.uint32)
    n_rolls = bm1.size
    if off is not None:
        off = np.ascontiguousarray(off, dtype=np.uint32)
        n_batches = off.size - 1
    else:
        n_batches = n_rolls
    out = np.zeros(n_rolls, dtype=np.uint32)
    _check(_load().orc_dice(_ptr(bm1), _ptr(off), n_batches, n_rolls, seed, _ptr(out)), "dice")
    return out


def dice_fixed(b: int, k: int, n_rolls: int, seed: int) -> np.ndarray:
    out = np.zeros(n_rolls, dtype=np.uint32)
    _check(_load().orc_dice_fixed(b, k, n_rolls, seed, _ptr(out)), "dice_fixed")
    return out


# ------------------------------------------------- threads over batches --
# The word of every batch is a function of (seed, batch index, attempt) only,
# so disjoint batch ranges (or independent arrays) can be rolled by separate
# host threads with results identical to the one-thread functions above.  The
# C calls release the GIL.


def host_threads() -> int:
    """Host cores available to this process."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _ranges(n: int, parts: int):
    parts = max(1, min(parts, n)) if n else 1
    step = (n + parts - 1) // parts
    return [(a, min(n, a + step)) for a in range(0, n, step)] if n else []


def dice_parallel(bm1: np.ndarray, off: np.ndarray | None, seed: int, threads: int | None = None,
                  chunks: int | None = None) -> np.ndarray:
    """orc_dice on `threads` host threads over contiguous batch ranges."""
    bm1 = np.ascontiguousarray(bm1, dtype=np.uint32)
    n_rolls = bm1.size
    lib = _load()
    if off is not None:
        off = np.ascontiguousarray(off, dtype=np.uint32)
        n_batches = off.size - 1
        if n_batches < 0 or off[0] != 0 or off[-1] != n_rolls or np.any(np.diff(off.astype(np.int64)) < 0):
            raise OracleError("dice_parallel: invalid CSR offsets")
    else:
        n_batches = n_rolls
    out = np.zeros(n_rolls, dtype=np.uint32)
    threads = threads or host_threads()

    def run(r):
        _check(lib.orc_dice_range(_ptr(bm1), _ptr(off), r[0], r[1], seed, _ptr(out)), "dice_range")

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, _ranges(n_batches, chunks or 4 * threads)))
    return out


def dice_fixed_parallel(b: int, k: int, n_rolls: int, seed: int, threads: int | None = None) -> np.ndarray:
    """orc_dice_fixed on `threads` host threads over contiguous batch ranges."""
    out = np.zeros(n_rolls, dtype=np.uint32)
    lib = _load()
    threads = threads or host_threads()
    n_batches = (n_rolls + k - 1) // k if k else 0

    def run(r):
        _check(lib.orc_dice_fixed_range(b, k, n_rolls, r[0], r[1], seed, _ptr(out)), "dice_fixed_range")

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, _ranges(n_batches, 4 * threads)))
    return out


def shuffle_batched_parallel(data: np.ndarray, offsets: np.ndarray, seeds: np.ndarray, nk=PAPER_NK,
                             k_max: int = PAPER_KMAX, threads: int | None = None) -> np.ndarray:
    """orc_shuffle_batched on `threads` host threads over ranges of arrays
    (balanced by element count)."""
    z = np.array(data, copy=True)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    n_arrays = seeds.size
    lib = _load()
    nka = _nk_array(nk)
    threads = threads or host_threads()
    parts = 8 * threads
    total = int(offsets[n_arrays]) if n_arrays else 0
    cuts = [0]
    for p in range(1, parts):
        c = int(np.searchsorted(offsets[: n_arrays + 1], total * p // parts, side="left"))
        cuts.append(min(max(c, cuts[-1]), n_arrays))
    cuts.append(n_arrays)
    spans = [(a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]

    def run(r):
        a, b = r
        _check(lib.orc_shuffle_batched(_ptr(z), _ptr(offsets[a: b + 1]), b - a, z.dtype.itemsize,
                                       _ptr(seeds[a:b]), _ptr(nka), k_max), "shuffle_batched")

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, spans))
    return z


# --------------------------------------------------------------- shuffles --
def k_rule(i: int, nk=PAPER_NK, k_max: int = PAPER_KMAX) -> int:
    return _load().orc_k_rule(i, _ptr(_nk_array(nk)), k_max)


def shuffle(data: np.ndarray, seed: int, nk=PAPER_NK, k_max: int = PAPER_KMAX):
    """Shuffle a copy of data (uint32 or uint64); returns (shuffled, j)."""
    z = np.array(data, copy=True)
    assert z.dtype in (np.uint32, np.uint64)
    j = np.zeros(z.size, dtype=np.uint32)
    _check(
        _load().orc_shuffle(_ptr(z), z.size, z.dtype.itemsize, seed, _ptr(_nk_array(nk)), k_max, _ptr(j)),
        "shuffle",
    )
    return z, j


def apply_swaps(data: np.ndarray, j: np.ndarray) -> np.ndarray:
    z = np.array(data, copy=True)
    j = np.ascontiguousarray(j, dtype=np.uint32)
    _check(_load().orc_apply_swaps(_ptr(z), z.size, z.dtype.itemsize, _ptr(j)), "apply_swaps")
    return z


def shuffle_batched(data: np.ndarray, offsets: np.ndarray, seeds: np.ndarray,
                    nk=PAPER_NK, k_max: int = PAPER_KMAX) -> np.ndarray:
    z = np.array(data, copy=True)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    _check(
        _load().orc_shuffle_batched(_ptr(z), _ptr(offsets), seeds.size, z.dtype.itemsize,
                                    _ptr(seeds), _ptr(_nk_array(nk)), k_max),
        "shuffle_batched",
    )
    return z


def sample(n: int, m: int, seed: int, nk=PAPER_NK, k_max: int = PAPER_KMAX) -> np.ndarray:
    out = np.zeros(m, dtype=np.uint32)
    _check(_load().orc_sample(n, m, seed, _ptr(_nk_array(nk)), k_max, _ptr(out)), "sample")
    return out


def partial_shuffle_word_L(L: int, z: np.ndarray, i: int, k: int, u: int, r0: int):
    """One Algorithm 4 step at word size L with an explicit word; z (uint64)
    is updated in place.  Returns (accepted, digits)."""
    assert z.dtype == np.uint64 and z.flags["C_CONTIGUOUS"]
    a = np.zeros(k, dtype=np.uint64)
    res = _load().orc_partial_shuffle_word_L(L, _ptr(z), i, k, u, r0, _ptr(a))
    if res < 0:
        raise OracleError("partial_shuffle_word_L: invalid input")
    return bool(res), [int(x) for x in a]


# ------------------------------------------------------------ cost model --
# the schedule of the paper's naive_shuffle_2: single dice while more than
# 2^32 elements remain, pairs below
NAIVE2_NK = (0, 0, 1 << 32, 0, 0, 0, 0, 0, 0)
NAIVE2_KMAX = 2


def naive_shuffle(data: np.ndarray, seed: int, nk=NAIVE2_NK, k_max: int = NAIVE2_KMAX):
    """The naive batched shuffle (division-based digits) of a copy of data;
    returns (shuffled, j)."""
    z = np.array(data, copy=True)
    assert z.dtype in (np.uint32, np.uint64)
    j = np.zeros(z.size, dtype=np.uint32)
    _check(_load().orc_naive_shuffle(_ptr(z), z.size, z.dtype.itemsize, seed, _ptr(_nk_array(nk)),
                                     k_max, _ptr(j)), "naive_shuffle")
    return z, j


def naive_digits(v: int, i: int, k: int) -> list[int]:
    d = np.zeros(k, dtype=np.uint64)
    _load().orc_naive_digits(v, i, k, _ptr(d))
    return [int(x) for x in d]


def cost_avg(k: int, n: int, L: int = 64, c_rng: float = 2.0, c_div: float = 16.0) -> float:
    return _load().orc_cost_avg(k, n, L, c_rng, c_div)


def nk(k: int, L: int = 64, c_rng: float = 2.0, c_div: float = 16.0, n_limit: int = 1 << 40) -> int:
    return _load().orc_nk(k, L, c_rng, c_div, n_limit)


# ----------------------------------------------------- other word sources --
# Counter-based alternatives to the SplitMix64 words (Section 7 compares
# generators of different cost): ChaCha20 blocks (L = 64) and the high half of
# the SplitMix64 word (L = 32).
SRC_SPLITMIX64, SRC_CHACHA20, SRC_SPLITMIX32 = 0, 1, 2

# Table 2's L = 32 estimates (20724, 581, 109) rounded down to powers of two,
# the reduction Section 6.1 applies to the L = 64 column.
L32_NK = (0, 0, 1 << 14, 1 << 9, 1 << 6, 0, 0, 0, 0)
L32_KMAX = 4


def chacha_block(inp, rounds: int = 20) -> np.ndarray:
    """The ChaCha block function on 16 uint32 words (input added back)."""
    inp = np.ascontiguousarray(inp, dtype=np.uint32)
    assert inp.size == 16
    out = np.zeros(16, dtype=np.uint32)
    _load().orc_chacha_block(_ptr(inp), rounds, _ptr(out))
    return out


def chacha_input(seed: int, c: int) -> np.ndarray:
    inp = np.zeros(16, dtype=np.uint32)
    _load().orc_chacha_input(seed, c, _ptr(inp))
    return inp


def src_bits(src: int) -> int:
    return _load().orc_src_bits(src)


def word_src(src: int, seed: int, g: int, a: int) -> int:
    return _load().orc_word_src(src, seed, g, a)


def roll_batch_src(src: int, b, seed: int, g: int):
    """Algorithm 3 with the words of source src: (digits, attempts used)."""
    b = np.ascontiguousarray(b, dtype=np.uint64)
    a = np.zeros(len(b), dtype=np.uint64)
    att = np.zeros(1, dtype=np.uint32)
    _check(_load().orc_roll_batch_src(src, _ptr(b), len(b), seed, g, _ptr(a), _ptr(att)), "roll_batch_src")
    return [int(x) for x in a], int(att[0])


def shuffle_src(src: int, data: np.ndarray | None, seed: int, nk=None, k_max: int | None = None, n: int | None = None):
    """Shuffle a copy of data with the words of source src; returns
    (shuffled or None, j).  With data None only the swap indices of an n-element
    shuffle are formed.  The default schedule is the paper's for L = 64 and
    L32_NK for L = 32."""
    if nk is None:
        nk, k_max = (L32_NK, L32_KMAX) if src == SRC_SPLITMIX32 else (PAPER_NK, PAPER_KMAX)
    z = None
    if data is not None:
        z = np.array(data, copy=True)
        assert z.dtype in (np.uint32, np.uint64)
        n = z.size
    j = np.zeros(n, dtype=np.uint32)
    eb = z.dtype.itemsize if z is not None else 4
    _check(_load().orc_shuffle_src(src, _ptr(z), n, eb, seed, _ptr(_nk_array(nk)), k_max, _ptr(j)),
           "shuffle_src")
    return z, j


def dice_fixed_src(src: int, b: int, k: int, n_rolls: int, seed: int) -> np.ndarray:
    """Algorithm 2 bulk dice of one bound with the words of source src."""
    out = np.zeros(n_rolls, dtype=np.uint32)
    _check(_load().orc_dice_fixed_src(src, b, k, n_rolls, seed, _ptr(out)), "dice_fixed_src")
    return out


def dice_src(src: int, bm1: np.ndarray, off: np.ndarray | None, seed: int) -> np.ndarray:
    """Per-roll-bound dice (Algorithm 3, CSR batches) with the words of source src."""
    bm1 = np.ascontiguousarray(bm1, dtype=np.uint32)
    n_rolls = bm1.size
    if off is not None:
        off = np.ascontiguousarray(off, dtype=np.uint32)
        n_batches = off.size - 1
    else:
        n_batches = n_rolls
    out = np.zeros(n_rolls, dtype=np.uint32)
    _check(_load().orc_dice_src(src, _ptr(bm1), _ptr(off) if off is not None else None, n_batches, n_rolls,
                                seed, _ptr(out)), "dice_src")
    return out
