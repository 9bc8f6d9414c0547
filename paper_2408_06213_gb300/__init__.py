"""brr -- batched ranged random integers and batched Fisher-Yates on GB300.

Thin Python binding over the libbrr C ABI (include/brr.h).  Device memory
and streams come from PyTorch; every computation runs in libbrr's CUDA
kernels.  Methods that receive device tensors queue work on the current (or
given) stream and return at once; methods that receive CPU tensors copy the
inputs to the device, run, copy the results back and synchronise (the
end-to-end form).
"""
from __future__ import annotations

import ctypes as C
import threading

import torch

from ._lib import (BRR_OK, SCHED_KMAX, Schedule, Segment, exported_symbols, lib)

__all__ = ["BrrError", "Context", "schedule", "naive_schedule", "l32_schedule", "plan", "default_context",
           "exported_symbols", "WORDS_SPLITMIX64", "WORDS_CHACHA20", "WORDS_SPLITMIX32"]

# counter-based word sources of Context.shuffle_words (brr_word_source)
WORDS_SPLITMIX64, WORDS_CHACHA20, WORDS_SPLITMIX32 = 0, 1, 2


class BrrError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = lib().brr_status_str(status).decode()
        super().__init__(f"{what}: {msg}")


def _check(st: int, what: str):
    if st != BRR_OK:
        raise BrrError(st, what)


def schedule(n_k: dict | None = None, k_max: int | None = None) -> Schedule:
    """A batch-size schedule.  Default: the paper's (n_2..n_6 = 2^30, 2^19,
    2^14, 2^11, 2^9, k_max = 6).  n_k maps k -> threshold and replaces the
    whole table; k_max alone caps the default table (k_max = 1: unbatched)."""
    s = Schedule()
    lib().brr_schedule_paper(C.byref(s))
    if n_k is not None:
        for k in range(SCHED_KMAX + 1):
            s.n_k[k] = int(n_k.get(k, 0))
        s.k_max = max([1] + [k for k in n_k if k >= 2])
    if k_max is not None:
        s.k_max = int(k_max)
    return s


def naive_schedule() -> Schedule:
    """The schedule of the paper's naive_shuffle_2 (pairs up to 2^32 remaining)."""
    s = Schedule()
    lib().brr_schedule_naive2(C.byref(s))
    return s


def l32_schedule() -> Schedule:
    """The L = 32 schedule (Table 2's L = 32 column rounded down to powers of
    two: n_2, n_3, n_4 = 2^14, 2^9, 2^6)."""
    s = Schedule()
    lib().brr_schedule_l32(C.byref(s))
    return s


def plan(n: int, stop: int = 1, sched: Schedule | None = None):
    """Host-side batch plan of a (partial) shuffle: (segments, n_batches)."""
    L = lib()
    ns, nb = C.c_uint32(0), C.c_uint64(0)
    sp = C.byref(sched) if sched is not None else None
    _check(L.brr_shuffle_plan(n, stop, sp, None, 0, C.byref(ns), C.byref(nb)), "plan")
    segs = (Segment * max(1, ns.value))()
    _check(L.brr_shuffle_plan(n, stop, sp, segs, ns.value, C.byref(ns), C.byref(nb)), "plan")
    out = [dict(g0=s.g0, count=s.count, u=s.u, i0=s.i0, k=s.k) for s in segs[: ns.value]]
    return out, nb.value


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_ptr(t: torch.Tensor | None, dtype, name: str, device):
    if t is None:
        return None
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_cuda or t.device != device:
        raise ValueError(f"{name}: expected a tensor on {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    return t.data_ptr()


_U32 = torch.uint32 if hasattr(torch, "uint32") else torch.int32
_U64 = torch.uint64 if hasattr(torch, "uint64") else torch.int64


def _as_u32(t: torch.Tensor) -> torch.Tensor:
    return t if t.dtype == _U32 else t.view(_U32) if t.element_size() == 4 else t


class Context:
    """A libbrr context bound to one CUDA device (owns scratch memory)."""

    def __init__(self, device: int | torch.device | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("brr needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().brr_create(C.byref(self._h)), "brr_create")

    def close(self):
        if self._h:
            lib().brr_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ errors --
    def check(self, stream=None):
        """Synchronise `stream` and raise if a kernel recorded an error."""
        _check(lib().brr_last_device_error(self._h, _stream_handle(stream)), "device")

    # how shuffles apply their swap sequence (same result, bit for bit)
    SWAP_AUTO, SWAP_ROUNDS, SWAP_CHAINS = 0, 1, 2

    def set_swap_method(self, method: int):
        """BRR_SWAP_ROUNDS (deterministic-reservation rounds), BRR_SWAP_CHAINS
        (chain resolution) or BRR_SWAP_AUTO (the library's choice)."""
        _check(lib().brr_set_swap_method(self._h, method), "brr_set_swap_method")

    # kernel routing of chain-resolution shuffles (brr_tune_param)
    TUNE_SINGLE_CTA_MAX, TUNE_SMALL_MAX, TUNE_MEDIUM_MAX, TUNE_GRID_COOPERATIVE, TUNE_FIXED_SWEEP = 1, 2, 3, 4, 5
    TUNE_ORDERED_PUSH = 6
    TUNE_WINDOW_ROUTE = 7

    def tune(self, param: int, value: int):
        _check(lib().brr_tune(self._h, param, value), "brr_tune")

    def tune_get(self, param: int) -> int:
        v = C.c_uint64()
        _check(lib().brr_tune_get(self._h, param, C.byref(v)), "brr_tune_get")
        return v.value

    def calibrate(self, stream=None) -> dict:
        """GPU nanoseconds per random word, chain step (one die) and exact
        threshold (B >= 2^48 and B < 2^40): the cost model's inputs."""
        ns = (C.c_double * 4)()
        with torch.cuda.device(self.device):
            _check(lib().brr_calibrate(self._h, ns, _stream_handle(stream)), "brr_calibrate")
        return {"word": ns[0], "step": ns[1], "threshold_large": ns[2], "threshold_small": ns[3]}

    def selftest_attempt_limit(self, limit: int):
        """Attempts a bulk-dice batch may use before BRR_ERETRY (test hook;
        2^16 restores the default)."""
        _check(lib().brr_selftest_attempt_limit(self._h, limit), "brr_selftest_attempt_limit")

    def selftest_barrier_timeout(self, limit_ns: int, stream=None) -> int:
        """Run the bounded grid barrier on a wait that cannot complete
        (brr_selftest_barrier_timeout); returns the device status it recorded
        (BRR_ETIMEOUT expected) after the work on `stream` has finished."""
        with torch.cuda.device(self.device):
            _check(lib().brr_selftest_barrier_timeout(self._h, limit_ns, _stream_handle(stream)),
                   "brr_selftest_barrier_timeout")
            return lib().brr_last_device_error(self._h, _stream_handle(stream))

    def reserve(self, max_shuffle_len: int, max_sample_m: int = 0):
        _check(lib().brr_reserve(self._h, max_shuffle_len, max_sample_m), "brr_reserve")

    # -------------------------------------------------------------- dice --
    def dice(self, bm1: torch.Tensor, off: torch.Tensor | None, seed: int,
             out: torch.Tensor | None = None, stream=None, sync: bool = True, source: int = 0) -> torch.Tensor:
        """Rolls with bounds bm1 + 1 (uint32) in CSR batches off (uint32;
        None = one roll per batch, the unbatched form).  With host tensors
        the copies in, the kernel and the copy out are queued on `stream`
        (default: the current stream); sync=False returns without waiting,
        so that calls on different streams overlap their copies (call
        check(stream) before reading `out`).  source: the word source
        (brr_dice_words; 0 = SplitMix64, brr_dice)."""
        if not bm1.is_cuda:
            s = self._stream(stream)
            d_bm1 = self._to_device("dice.bm1", bm1, s)
            d_off = self._to_device("dice.off", off, s) if off is not None else None
            d_out = self._staging("dice.out", bm1.numel(), _U32, s)
            self.dice(d_bm1, d_off, seed, out=d_out, stream=s, source=source)
            return self._to_host(d_out, out, s, sync)
        n_rolls = bm1.numel()
        n_batches = off.numel() - 1 if off is not None else n_rolls
        if out is None:
            out = torch.empty(n_rolls, dtype=_U32, device=bm1.device)
        bp = _dev_ptr(_as_u32(bm1), _U32, "bm1", self.device)
        opp = _dev_ptr(_as_u32(off), _U32, "off", self.device) if off is not None else None
        outp = _dev_ptr(out, _U32, "out", self.device)
        with torch.cuda.device(self.device):
            if source == WORDS_SPLITMIX64:
                st = lib().brr_dice(self._h, bp, opp, n_batches, n_rolls, seed, outp, _stream_handle(stream))
            else:
                st = lib().brr_dice_words(self._h, source, bp, opp, n_batches, n_rolls, seed, outp,
                                          _stream_handle(stream))
            _check(st, "brr_dice")
        return out

    def dice_fixed(self, b: int, k: int, n_rolls: int, seed: int,
                   out: torch.Tensor | None = None, stream=None, source: int = 0,
                   sync: bool = True) -> torch.Tensor:
        """Rolls in [0, b), k per word (brr_dice_fixed; brr_dice_fixed_words
        for another word source).  A host `out` is filled as in dice()."""
        if out is not None and not out.is_cuda:
            s = self._stream(stream)
            d_out = self._staging("dice_fixed.out", n_rolls, _U32, s)
            self.dice_fixed(b, k, n_rolls, seed, out=d_out, stream=s, source=source)
            return self._to_host(d_out, out, s, sync)
        if out is None:
            out = torch.empty(n_rolls, dtype=_U32, device=self.device)
        op = _dev_ptr(out, _U32, "out", self.device)
        with torch.cuda.device(self.device):
            if source == WORDS_SPLITMIX64:
                st = lib().brr_dice_fixed(self._h, b, k, n_rolls, seed, op, _stream_handle(stream))
            else:
                st = lib().brr_dice_fixed_words(self._h, source, b, k, n_rolls, seed, op, _stream_handle(stream))
            _check(st, "brr_dice_fixed")
        return out

    # ---------------------------------------------------------- shuffles --
    def shuffle(self, data: torch.Tensor, seed: int, sched: Schedule | None = None,
                j_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Shuffle data (4- or 8-byte elements) in place; returns data."""
        if not data.is_cuda:
            s = self._stream(stream)
            d = self._to_device("shuffle.data", data, s)
            self.shuffle(d, seed, sched=sched, stream=s)
            return self._to_host(d, data, s)
        if not data.is_contiguous() or data.device != self.device:
            raise ValueError("data: contiguous tensor on the context's device expected")
        eb = data.element_size()
        with torch.cuda.device(self.device):
            _check(lib().brr_shuffle(self._h, data.data_ptr(), data.numel(), eb, seed,
                                     C.byref(sched) if sched is not None else None,
                                     _dev_ptr(j_out, _U32, "j_out", self.device),
                                     _stream_handle(stream)), "brr_shuffle")
        return data

    def swap_indices(self, n: int, seed: int, sched: Schedule | None = None, naive: bool = False,
                     j_out: torch.Tensor | None = None, stream=None, source: int = 0) -> torch.Tensor:
        """Only the swap indices j[] of a shuffle of n elements (brr_shuffle,
        brr_shuffle_naive with naive=True, or brr_shuffle_words with another
        word source; data NULL)."""
        if j_out is None:
            j_out = torch.empty(max(n, 1), dtype=_U32, device=self.device)[:n]
        sp = C.byref(sched) if sched is not None else None
        jp = _dev_ptr(j_out, _U32, "j_out", self.device)
        with torch.cuda.device(self.device):
            if source != WORDS_SPLITMIX64:
                if naive:
                    raise ValueError("the naive method uses the SplitMix64 words only")
                st = lib().brr_shuffle_words(self._h, source, None, n, 4, seed, sp, jp, _stream_handle(stream))
            else:
                fn = lib().brr_shuffle_naive if naive else lib().brr_shuffle
                st = fn(self._h, None, n, 4, seed, sp, jp, _stream_handle(stream))
            _check(st, "swap indices")
        return j_out

    def shuffle_words(self, data: torch.Tensor, seed: int, source: int, sched: Schedule | None = None,
                      j_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Shuffle data in place with the words of `source` (WORDS_SPLITMIX64,
        WORDS_CHACHA20 or WORDS_SPLITMIX32; sched None = that source's default
        schedule); returns data."""
        if not data.is_contiguous() or not data.is_cuda or data.device != self.device:
            raise ValueError("data: contiguous tensor on the context's device expected")
        with torch.cuda.device(self.device):
            _check(lib().brr_shuffle_words(self._h, source, data.data_ptr(), data.numel(), data.element_size(),
                                           seed, C.byref(sched) if sched is not None else None,
                                           _dev_ptr(j_out, _U32, "j_out", self.device),
                                           _stream_handle(stream)), "brr_shuffle_words")
        return data

    def shuffle_naive(self, data: torch.Tensor, seed: int, sched: Schedule | None = None,
                      j_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """The paper's naive batched shuffle (one roll of each batch's product,
        digits by division; sched None = pairs, naive_shuffle_2), in place."""
        if not data.is_contiguous() or not data.is_cuda or data.device != self.device:
            raise ValueError("data: contiguous tensor on the context's device expected")
        with torch.cuda.device(self.device):
            _check(lib().brr_shuffle_naive(self._h, data.data_ptr(), data.numel(), data.element_size(), seed,
                                           C.byref(sched) if sched is not None else None,
                                           _dev_ptr(j_out, _U32, "j_out", self.device),
                                           _stream_handle(stream)), "brr_shuffle_naive")
        return data

    def shuffle_batched(self, data: torch.Tensor, offsets: torch.Tensor, seeds: torch.Tensor,
                        max_len: int, sched: Schedule | None = None, stream=None, source: int = 0) -> torch.Tensor:
        """Shuffle every array of data (CSR offsets, one seed each) in place;
        source: the word source (brr_shuffle_batched_words; 0 = SplitMix64)."""
        if not data.is_cuda:
            s = self._stream(stream)
            d = self._to_device("batched.data", data, s)
            self.shuffle_batched(d, self._to_device("batched.off", offsets, s),
                                 self._to_device("batched.seeds", seeds, s), max_len, sched, s, source)
            return self._to_host(d, data, s)
        n_arrays = seeds.numel()
        op = _dev_ptr(offsets, _U64, "offsets", self.device)
        sp = _dev_ptr(seeds, _U64, "seeds", self.device)
        sc = C.byref(sched) if sched is not None else None
        with torch.cuda.device(self.device):
            if source == WORDS_SPLITMIX64:
                st = lib().brr_shuffle_batched(self._h, data.data_ptr(), op, n_arrays, data.element_size(), sp,
                                               max_len, sc, _stream_handle(stream))
            else:
                st = lib().brr_shuffle_batched_words(self._h, source, data.data_ptr(), op, n_arrays,
                                                     data.element_size(), sp, max_len, sc, _stream_handle(stream))
            _check(st, "brr_shuffle_batched")
        return data

    # ----------------------------------------------------------- samples --
    def sample(self, n: int, m: int, seed: int, sched: Schedule | None = None,
               out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(m, dtype=_U32, device=self.device)
        with torch.cuda.device(self.device):
            _check(lib().brr_sample(self._h, n, m, seed, C.byref(sched) if sched is not None else None,
                                    _dev_ptr(out, _U32, "out", self.device), _stream_handle(stream)),
                   "brr_sample")
        return out

    def sample_batched(self, n: torch.Tensor, m: torch.Tensor, seeds: torch.Tensor,
                       out_off: torch.Tensor, max_m: int, out: torch.Tensor,
                       sched: Schedule | None = None, stream=None) -> torch.Tensor:
        with torch.cuda.device(self.device):
            _check(lib().brr_sample_batched(self._h, _dev_ptr(n, _U64, "n", self.device),
                                            _dev_ptr(_as_u32(m), _U32, "m", self.device),
                                            _dev_ptr(seeds, _U64, "seeds", self.device),
                                            _dev_ptr(out_off, _U64, "out_off", self.device),
                                            seeds.numel(), max_m,
                                            C.byref(sched) if sched is not None else None,
                                            _dev_ptr(out, _U32, "out", self.device),
                                            _stream_handle(stream)), "brr_sample_batched")
        return out

    # --------------------------------------------------- end-to-end form --
    def _stream(self, stream):
        """The torch stream host-buffer forms queue on."""
        if stream is None:
            return torch.cuda.current_stream(self.device)
        return stream

    def _staging(self, key: str, numel: int, dtype, stream) -> torch.Tensor:
        """A reusable device buffer for the host-buffer forms, one per key and
        stream (work on one stream reuses it in stream order; work on
        different streams never shares it)."""
        if not hasattr(self, "_stage"):
            self._stage = {}
        sk = (key, _stream_handle(stream))
        t = self._stage.get(sk)
        if t is None or t.numel() < numel or t.dtype != dtype:
            t = torch.empty(numel, dtype=dtype, device=self.device)
            self._stage[sk] = t
        return t[:numel]

    def _to_device(self, key: str, t: torch.Tensor, stream) -> torch.Tensor:
        d = self._staging(key, t.numel(), t.dtype, stream)
        with torch.cuda.stream(stream):
            d.copy_(t.reshape(-1), non_blocking=True)
        return d

    def _to_host(self, d: torch.Tensor, out: torch.Tensor | None, stream, sync: bool = True) -> torch.Tensor:
        """Copy a device result to `out` (or a new pinned tensor) on `stream`;
        with sync, wait for it and raise any device-side error."""
        if out is None:
            out = torch.empty(d.shape, dtype=d.dtype, pin_memory=True)
        with torch.cuda.stream(stream):
            out.reshape(-1).copy_(d, non_blocking=True)
        if sync:
            self.check(stream)
        return out


_tls = threading.local()


def default_context() -> Context:
    """One context per host thread and device."""
    dev = torch.cuda.current_device()
    ctxs = getattr(_tls, "ctxs", None)
    if ctxs is None:
        ctxs = _tls.ctxs = {}
    if dev not in ctxs:
        ctxs[dev] = Context(dev)
    return ctxs[dev]
