"""Continuous-batching server for shuffle and sample requests on one GPU.

Requests arrive over time: full shuffles (a random permutation of the n
elements 0..n-1, produced on the device) and partial Fisher-Yates samples
(m distinct values from [0, n)).  The engine keeps a pool of slots, each a
CUDA stream with its own brr context (so that scratch memory is never shared
between work in flight).  Whenever a slot is free it admits the waiting
requests in arrival order while their device memory fits the budget, and
launches them as one wave: one `brr_shuffle_batched` launch for the
shuffles that fit one thread-block cluster's shared memory, one
`brr_shuffle` call (grid-wide path) per longer shuffle, and one
`brr_sample_batched` launch for the samples.  Requests that
arrive while earlier waves run are admitted into the next wave on another
slot, so waves overlap on the device; a request leaves when its wave's
completion event has fired.

Every request's result depends only on its own (kind, n, m, seed): the same
alone and in any mix.  A request without a seed gets base_seed + its id; the
word generator's counters (batch index, attempt) exist only inside the
kernels, so no generator state ever moves between host and device.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import Context

SHUFFLE, SAMPLE = 0, 1
STAGED_CAP = 65536  # longest shuffle staged in one thread-block cluster


@dataclasses.dataclass
class Request:
    rid: int
    kind: int
    n: int
    m: int = 0
    seed: int | None = None
    arrival: float = 0.0          # seconds on the engine clock
    admitted: float = -1.0
    done: float = -1.0
    result: torch.Tensor | None = None  # device tensor (n values, or m values)

    @property
    def elements(self) -> int:
        return self.n if self.kind == SHUFFLE else self.m

    def device_bytes(self) -> int:
        """Device memory the request holds while its wave runs: a shuffle's
        uint32 result plus the int32 start offsets used to build its identity
        array (batched path), a sample's uint32 result, and per-request
        metadata.  Context scratch is reserved once per slot at start-up and is
        not part of the budget."""
        if self.kind == SHUFFLE:
            return 8 * self.n + 64
        return 4 * self.m + 64


class _Slot:
    def __init__(self, device, swap_method: int | None, grid_cooperative: bool, max_n: int, max_m: int):
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = Context(device)
        if swap_method is not None:
            self.ctx.set_swap_method(swap_method)
        # a cooperative launch needs the whole GPU; the slots share it
        self.ctx.tune(Context.TUNE_GRID_COOPERATIVE, 1 if grid_cooperative else 0)
        # scratch for the largest request, once: growing it while serving
        # would allocate and synchronise the device, stalling every slot
        self.ctx.reserve(max_n, max_m)
        self.event = None
        self.wave: list[Request] = []
        self.bytes = 0
        self.keep = []  # tensors that must live until the wave completes


class ServeEngine:
    """Continuous batching over `n_slots` streams with an HBM admission budget."""

    def __init__(self, device: int = 0, n_slots: int = 4, hbm_budget: int | None = None,
                 max_wave: int = 8192, base_seed: int = 0x5EED, swap_method: int | None = None,
                 grid_cooperative: bool = False, max_n: int = 10 ** 7, max_m: int = 10 ** 4):
        """max_n / max_m: the largest shuffle and sample accepted; every slot
        reserves its scratch for them at start-up.  hbm_budget: device bytes
        that admitted requests may hold at once (default: half of the memory
        still free after the slots' scratch is reserved)."""
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.max_n, self.max_m = int(max_n), int(max_m)
        self.slots = [_Slot(self.device, swap_method, grid_cooperative, self.max_n, self.max_m)
                      for _ in range(n_slots)]
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(free * 0.5)
        self.hbm_budget = hbm_budget
        self.in_use = 0
        self.max_wave = max_wave
        self.max_in_flight = 0  # most waves launched and not yet finished when one starts
        self.wave_events = []   # (start, end) timing events of every wave, in launch order
        self.base_seed = base_seed
        self.waiting: collections.deque[Request] = collections.deque()
        self.finished: list[Request] = []
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ------------------------------------------------------------- admission --
    def submit(self, req: Request):
        if (req.kind == SHUFFLE and req.n > self.max_n) or (req.kind == SAMPLE and req.m > self.max_m):
            raise ValueError(f"request {req.rid} is larger than the engine's reserved limits "
                             f"(n <= {self.max_n}, m <= {self.max_m})")
        self.waiting.append(req)

    def _admit(self, slot: _Slot) -> list[Request]:
        wave, budget_left = [], self.hbm_budget - self.in_use
        while self.waiting and len(wave) < self.max_wave:
            r = self.waiting[0]
            b = r.device_bytes()
            if b > budget_left:
                if not wave and self.in_use == 0:
                    raise RuntimeError(f"request {r.rid} needs {b} bytes, above the whole budget")
                break
            self.waiting.popleft()
            budget_left -= b
            wave.append(r)
        return wave

    def _launch(self, slot: _Slot, wave: list[Request]):
        t = self.now()
        for r in wave:
            r.admitted = t
        dev = self.device
        keep = []
        with torch.cuda.stream(slot.stream):
            ev_start = torch.cuda.Event(enable_timing=True)
            ev_start.record(slot.stream)
            # seeds: a request without one takes base_seed + its id; the
            # generator's counters (batch, attempt) never leave the kernels
            for r in wave:
                if r.seed is None:
                    r.seed = (self.base_seed + r.rid) & 0xFFFFFFFFFFFFFFFF
            seeds_np = np.array([r.seed for r in wave], dtype=np.uint64)
            seeds_all = torch.from_numpy(seeds_np.view(np.int64)).to(dev, non_blocking=True)
            sh = [i for i, r in enumerate(wave) if r.kind == SHUFFLE]
            sa = [i for i, r in enumerate(wave) if r.kind == SAMPLE]
            # shuffles longer than one cluster's shared memory run one by one
            # on the grid-wide path; the rest go in one batched launch
            big = [i for i in sh if wave[i].n > STAGED_CAP]
            sh = [i for i in sh if wave[i].n <= STAGED_CAP]
            for i in big:
                r = wave[i]
                data_b = torch.arange(r.n, dtype=torch.int32, device=dev).view(torch.uint32)
                slot.ctx.shuffle(data_b, r.seed, stream=slot.stream)
                r.result = data_b
                keep.append(data_b)
            if sh:
                sizes = np.array([wave[i].n for i in sh], dtype=np.int64)
                off = np.zeros(len(sh) + 1, dtype=np.int64)
                np.cumsum(sizes, out=off[1:])
                off_d = torch.from_numpy(off).to(dev, non_blocking=True)
                total = int(off[-1])
                # identity arrays 0..n-1 side by side (int32: 4 bytes per
                # element for the array and 4 for its start offsets)
                data = torch.arange(total, dtype=torch.int32, device=dev)
                starts = torch.repeat_interleave(off_d[:-1].to(torch.int32), torch.from_numpy(sizes).to(dev),
                                                 output_size=total)
                data.sub_(starts)
                del starts
                data = data.view(torch.uint32)
                sh_idx = torch.tensor(sh, device=dev)
                s_sh = seeds_all[sh_idx].contiguous().view(torch.uint64)
                slot.ctx.shuffle_batched(data, off_d.view(torch.uint64), s_sh,
                                         int(sizes.max()), stream=slot.stream)
                keep.append(s_sh)
                for j, i in enumerate(sh):
                    wave[i].result = data[int(off[j]):int(off[j + 1])]
                keep += [data, off_d]
            if sa:
                ns = np.array([wave[i].n for i in sa], dtype=np.uint64)
                ms = np.array([wave[i].m for i in sa], dtype=np.uint32)
                oo = np.zeros(len(sa) + 1, dtype=np.uint64)
                np.cumsum(ms, out=oo[1:])
                out = torch.empty(max(1, int(oo[-1])), dtype=torch.uint32, device=dev)
                sa_idx = torch.tensor(sa, device=dev)
                n_d = torch.from_numpy(ns).to(dev)
                m_d = torch.from_numpy(ms).to(dev)
                o_d = torch.from_numpy(oo[:-1].copy()).to(dev)
                s_d = seeds_all[sa_idx].contiguous().view(torch.uint64)
                slot.ctx.sample_batched(n_d, m_d, s_d, o_d, int(ms.max()), out, stream=slot.stream)
                for j, i in enumerate(sa):
                    wave[i].result = out[int(oo[j]):int(oo[j + 1])]
                keep += [out, n_d, m_d, o_d, s_d]
            keep.append(seeds_all)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(slot.stream)
        self.wave_events.append((ev_start, ev))
        # waves of other slots still running on the device as this one starts
        others = sum(1 for o in self.slots if o is not slot and o.event is not None and not o.event.query())
        self.max_in_flight = max(self.max_in_flight, 1 + others)
        slot.event = ev
        slot.wave = wave
        slot.keep = keep
        slot.bytes = sum(r.device_bytes() for r in wave)
        self.in_use += slot.bytes

    def _retire(self, slot: _Slot):
        t = self.now()
        slot.ctx.check(slot.stream)
        for r in slot.wave:
            r.done = t
        self.finished.extend(slot.wave)
        self.in_use -= slot.bytes
        slot.wave, slot.event, slot.bytes, slot.keep = [], None, 0, []

    # ------------------------------------------------------------------ loop --
    def step(self) -> bool:
        """Retire finished waves, launch new ones; True if anything happened."""
        busy = False
        for s in self.slots:
            if s.event is not None and s.event.query():
                self._retire(s)
                busy = True
        for s in self.slots:
            if s.event is None and self.waiting:
                wave = self._admit(s)
                if wave:
                    self._launch(s, wave)
                    busy = True
        return busy

    def drain(self):
        while self.waiting or any(s.event is not None for s in self.slots):
            if not self.step():
                time.sleep(20e-6)

    def run_trace(self, arrivals, kinds, ns, ms, seeds=None, realtime: bool = True) -> dict:
        """Feed a request trace (arrival times in seconds) and serve it."""
        reqs = [Request(i, int(kinds[i]), int(ns[i]), int(ms[i]),
                        None if seeds is None else int(seeds[i]), float(arrivals[i]))
                for i in range(len(arrivals))]
        self.t0 = time.perf_counter()
        nxt = 0
        while nxt < len(reqs) or self.waiting or any(s.event is not None for s in self.slots):
            t = self.now()
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= t):
                if not realtime:
                    reqs[nxt].arrival = t
                self.submit(reqs[nxt])
                nxt += 1
            if not self.step():
                time.sleep(10e-6)
        for s in self.slots:
            torch.cuda.current_stream().wait_stream(s.stream)
        torch.cuda.synchronize(self.device)
        device_overlap = self.device_overlap()
        lat = np.array([r.done - r.arrival for r in reqs])
        span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
        elems = sum(r.elements for r in reqs)
        return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "elements": elems,
                "elements_per_s": elems / span, "span_s": span, "max_waves_in_flight": self.max_in_flight,
                "device_max_concurrent_waves": device_overlap, "waves": len(self.wave_events),
                "requests_list": reqs}

    def device_overlap(self) -> int:
        """Most waves whose device intervals (from the start event to the end
        event recorded on their slot's stream) overlap at one instant: a wave
        counts from the moment the device reaches its first queued operation
        until its last one has run.  Needs every wave finished."""
        if not self.wave_events:
            return 0
        ref = self.wave_events[0][0]
        marks = []
        for s, e in self.wave_events:
            marks.append((ref.elapsed_time(s), 1))
            marks.append((ref.elapsed_time(e), -1))
        marks.sort(key=lambda x: (x[0], x[1]))  # an end before a start at the same time
        cur = best = 0
        for _, d in marks:
            cur += d
            best = max(best, cur)
        return best
