"""Continuous-batching trigger request loop over the C ABI.

Events arrive one by one (a Poisson trace).  The scheduler keeps up to
`slots` micro-batches in flight on the device, each on its own CUDA stream
and its own ht_ctx (so their kernels overlap), and admits newly arrived
events into the next micro-batch as soon as a slot is free and the
accumulator memory of all in-flight batches stays within the budget.  Hits
are packed into pinned host buffers, copied to the device on the slot's
stream, processed by ht_process (vote, peaks, association) and the results
copied back; an event's latency runs from its arrival to the moment its
results are in host memory.

The scheduling logic is independent of the executor: `GpuExecutor` runs the
library, tests drive the same `Scheduler` with a fake executor on the CPU.
"""

from __future__ import annotations

import dataclasses
import json
import time
from typing import Callable, List, Optional, Sequence

import numpy as np

from . import synth


@dataclasses.dataclass
class Event:
    eid: int
    arrival: float             # seconds on the trace clock
    x: np.ndarray
    y: np.ndarray
    layer: np.ndarray


@dataclasses.dataclass
class EventResult:
    """Completion record of one event.  The peak list and CSR rows are in host
    memory when it is produced; they reach callers through the executor's
    `consumer(eid, peaks, offsets, hits, hit_base)` callback as views into the
    slot's pinned buffers, valid only during the callback (copy what you keep):
    peaks int32 [n, 5] (event, i_phi, i_d0, i_kappa, votes), offsets int64
    [n + 1] CSR pointers (absolute, subtract offsets[0]), hits int32 batch hit
    indices (subtract hit_base for indices within the event)."""

    eid: int
    n_peaks: int
    n_pairs: int


def poisson_trace(rate_hz: float, n_events: int, seed: int = 4, workload: str = "serving_lognormal"):
    """n_events arrivals at `rate_hz` with the workload's event sizes."""
    w = synth.WORKLOADS[workload]
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_events))
    batch = synth.generate(w, n_events=n_events, seed=seed)
    evs = []
    for e in range(n_events):
        lo, hi = int(batch.event_offsets[e]), int(batch.event_offsets[e + 1])
        evs.append(Event(e, float(t[e]), batch.x[lo:hi], batch.y[lo:hi], batch.layer[lo:hi]))
    return evs


class Scheduler:
    """Admission and continuous batching, independent of how batches run.

    executor must provide: slots (int), bytes_per_event (int),
    submit(slot, events) -> None, poll(slot) -> Optional[list[EventResult]]
    (None while running).
    """

    def __init__(self, executor, budget_bytes: int, max_batch: int, clock: Callable[[], float] = time.perf_counter):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.clock = clock
        if self.ex.bytes_per_event > self.budget:
            raise ValueError("one event's accumulator exceeds the memory budget")
        self.inflight = {}          # slot -> (events, bytes)
        self.pending: List[Event] = []
        self.done = {}              # eid -> (EventResult, completion time)
        self.max_inflight_bytes = 0
        self.batches = []           # (slot, n_events, submit time)

    def in_use(self) -> int:
        return sum(b for _, b in self.inflight.values())

    def admit(self, now: float):
        """Form micro-batches from arrived events while slots and memory allow."""
        for slot in range(self.ex.slots):
            if not self.pending:
                return
            if slot in self.inflight:
                continue
            room = (self.budget - self.in_use()) // self.ex.bytes_per_event
            n = min(len(self.pending), self.max_batch, room)
            if n <= 0:
                return
            evs, self.pending = self.pending[:n], self.pending[n:]
            b = n * self.ex.bytes_per_event
            self.inflight[slot] = (evs, b)
            self.max_inflight_bytes = max(self.max_inflight_bytes, self.in_use())
            self.batches.append((slot, n, now))
            self.ex.submit(slot, evs)

    def reap(self):
        for slot in list(self.inflight):
            out = self.ex.poll(slot)
            if out is None:
                continue
            t = self.clock()
            for r in out:
                self.done[r.eid] = (r, t)
            del self.inflight[slot]

    def run(self, events: Sequence[Event], t0: Optional[float] = None, timeout_s: float = 600.0):
        """Replay the trace in real time; returns {eid: (result, completion time - t0)}."""
        events = sorted(events, key=lambda e: e.arrival)
        t0 = self.clock() if t0 is None else t0
        i = 0
        deadline = t0 + timeout_s
        while len(self.done) < len(events):
            now = self.clock()
            if now > deadline:
                raise TimeoutError(f"trace not finished after {timeout_s} s")
            while i < len(events) and events[i].arrival <= now - t0:
                self.pending.append(events[i])
                i += 1
            self.reap()
            self.admit(now)
            if not self.inflight and not self.pending and i < len(events):
                # idle until the next arrival
                time.sleep(max(0.0, min(1e-3, events[i].arrival - (self.clock() - t0))))
        return {eid: (r, t - t0) for eid, (r, t) in self.done.items()}


def latency_stats(events: Sequence[Event], done) -> dict:
    lat = np.array([done[e.eid][1] - e.arrival for e in events])
    first = min(e.arrival for e in events)
    last = max(done[e.eid][1] for e in events)
    return {"events": len(events), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3),
            "throughput_eps": len(events) / max(last - first, 1e-9)}


class GpuExecutor:
    """Runs micro-batches through libht: one ht_ctx and CUDA stream per slot."""

    def __init__(self, grid, layer_r, threshold: int, window: int, slots: int = 3, max_batch: int = 512,
                 max_hits: int = 1 << 22, peak_cap: int = 1 << 24, pair_cap: int = 1 << 29, device=None,
                 copy_hits_back: bool = True, consumer=None):
        import torch

        from . import ht
        self.torch, self.ht = torch, ht
        self.dev = torch.device("cuda") if device is None else device
        self.thr, self.win = int(threshold), int(window)
        self.slots = int(slots)
        self.bytes_per_event = 4 * grid.n_phi * grid.n_d0 * grid.n_kappa
        self.copy_hits_back = copy_hits_back
        self.consumer = consumer
        self.state = []
        for _ in range(self.slots):
            ctx = ht.Context(grid, layer_r)
            ctx.set_option(ht.HT_OPT_USE_GRAPH, 0)  # batch shapes change every time
            st = {
                "ctx": ctx,
                "stream": torch.cuda.Stream(self.dev),
                "x": torch.empty(max_hits, dtype=torch.float32).pin_memory(),
                "y": torch.empty(max_hits, dtype=torch.float32).pin_memory(),
                "l": torch.empty(max_hits, dtype=torch.int8).pin_memory(),
                "o": torch.empty(max_batch + 1, dtype=torch.int32).pin_memory(),
                "res": ht.Results(peak_cap, pair_cap, device=self.dev),
                "h_peaks": torch.empty((peak_cap, 5), dtype=torch.int32).pin_memory(),
                "h_off": torch.empty(peak_cap + 1, dtype=torch.int64).pin_memory(),
                "h_hits": torch.empty(pair_cap, dtype=torch.int32).pin_memory(),
                "h_cnt": torch.empty(2, dtype=torch.int64).pin_memory(),
                "done": None, "events": None, "offs": None,
            }
            self.state.append(st)
        self.max_hits, self.max_batch = max_hits, max_batch
        self._reserve()

    def _reserve(self):
        """One batch of max_batch events holding max_hits hits (all at the
        origin) per slot, so that every device buffer of the slot's context
        reaches its largest size before the first request: growing a buffer
        later would free and allocate device memory, which synchronises the
        whole device in the middle of the trace."""
        ht = self.ht
        for st in self.state:
            st["x"].zero_()
            st["y"].zero_()
            st["l"].zero_()
            offs = np.linspace(0, self.max_hits, self.max_batch + 1).astype(np.int32)
            st["o"].numpy()[: self.max_batch + 1] = offs
            hits = ht.Hits.__new__(ht.Hits)
            hits.arrays = (st["x"], st["y"], st["o"], st["l"])
            hits.struct = ht.HtHits(st["x"].data_ptr(), st["y"].data_ptr(), None, st["l"].data_ptr(),
                                    st["o"].data_ptr(), self.max_batch, ht.HT_HOST, self.max_hits)
            st["ctx"].process(hits, self.thr, self.win, st["res"], st["stream"])
            try:
                st["ctx"].sync()
            except ht.HtError as e:
                if e.status != ht.HT_ERR_OVERFLOW:
                    raise

    def submit(self, slot, events):
        torch, ht = self.torch, self.ht
        st = self.state[slot]
        offs = np.zeros(len(events) + 1, np.int64)
        offs[1:] = np.cumsum([e.x.shape[0] for e in events])
        n = int(offs[-1])
        if n > self.max_hits or len(events) > self.max_batch:
            raise ValueError("micro-batch exceeds the executor's buffers")
        xs = st["x"].numpy()
        ys = st["y"].numpy()
        ls = st["l"].numpy()
        for e, a in zip(events, offs[:-1]):
            m = e.x.shape[0]
            xs[a:a + m], ys[a:a + m], ls[a:a + m] = e.x, e.y, e.layer
        st["o"].numpy()[: len(events) + 1] = offs
        hits = ht.Hits.__new__(ht.Hits)
        hits.arrays = (st["x"], st["y"], st["o"], st["l"])
        hits.struct = ht.HtHits(st["x"].data_ptr(), st["y"].data_ptr(), None, st["l"].data_ptr(),
                                st["o"].data_ptr(), len(events), ht.HT_HOST, n)
        s = st["stream"]
        st["ctx"].process(hits, self.thr, self.win, st["res"], s)
        with torch.cuda.stream(s):
            st["h_cnt"].copy_(st["res"].counts, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        st.update(done=ev, events=events, offs=offs, stage=1)

    def poll(self, slot):
        torch = self.torch
        st = self.state[slot]
        if not st["done"].query():
            return None
        if st["stage"] == 1:
            # counts are on the host: copy exactly the results back
            st["ctx"].sync()
            npk, npr = (int(v) for v in st["h_cnt"].numpy())
            s = st["stream"]
            with torch.cuda.stream(s):
                st["h_peaks"][:npk].copy_(st["res"].peaks[:npk], non_blocking=True)
                st["h_off"][: npk + 1].copy_(st["res"].peak_offsets[: npk + 1], non_blocking=True)
                if self.copy_hits_back:
                    st["h_hits"][:npr].copy_(st["res"].hit_idx[:npr], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s)
            st.update(done=ev, stage=2, npk=npk, npr=npr)
            if not ev.query():
                return None
        return self._unpack(st)

    def _unpack(self, st):
        npk = st["npk"]
        pk = st["h_peaks"][:npk].numpy()
        off = st["h_off"][: npk + 1].numpy()
        hits = st["h_hits"][: st["npr"]].numpy() if self.copy_hits_back else None
        offs = st["offs"]
        ev_col = pk[:, 0] if npk else np.zeros(0, np.int32)
        bounds = np.searchsorted(ev_col, np.arange(len(st["events"]) + 1))
        out = []
        for b, e in enumerate(st["events"]):
            lo, hi = int(bounds[b]), int(bounds[b + 1])
            if self.consumer is not None:
                self.consumer(e.eid, pk[lo:hi], off[lo:hi + 1],
                              None if hits is None else hits[off[lo]:off[hi]], int(offs[b]))
            out.append(EventResult(e.eid, hi - lo, int(off[hi] - off[lo])))
        st["done"] = None
        return out

    def close(self):
        for st in self.state:
            st["ctx"].close()


def measure(rates, n_events=4000, slots=3, max_batch=256, budget_gb=40.0, pair_cap=1 << 28, peak_cap=1 << 23,
            max_hits=1 << 21):
    """p50/p99 latency and throughput of the trigger loop at each offered load."""
    w = synth.WORKLOADS["serving_lognormal"]
    ex = GpuExecutor(w.grid, w.spec.layers, w.threshold, w.window, slots=slots, max_batch=max_batch,
                     max_hits=max_hits, peak_cap=peak_cap, pair_cap=pair_cap)
    out = []
    try:
        for rate in rates:
            evs = poisson_trace(float(rate), n_events)
            sch = Scheduler(ex, int(budget_gb * 2 ** 30), max_batch)
            done = sch.run(evs)
            st = latency_stats(evs, done)
            st.update(offered_eps=float(rate), slots=slots, max_batch=max_batch, batches=len(sch.batches),
                      mean_batch=float(np.mean([b[1] for b in sch.batches])),
                      max_inflight_gb=sch.max_inflight_bytes / 2 ** 30)
            out.append(st)
    finally:
        ex.close()
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="continuous-batching trigger loop at offered loads")
    ap.add_argument("--rates", default="20000,50000,100000,200000")
    ap.add_argument("--events", type=int, default=4000)
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    args = ap.parse_args(argv)
    for st in measure([float(r) for r in args.rates.split(",")], args.events, args.slots, args.max_batch,
                      args.budget_gb):
        print(json.dumps(st), flush=True)


if __name__ == "__main__":
    main()
