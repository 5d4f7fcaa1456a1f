"""Continuous-batching trigger loop.

CPU: the scheduler's admission, batching and latency accounting with a fake
executor.  GPU: every event's result is the same whether it ran alone or
inside a mixed, overlapping micro-batch.
"""

import numpy as np
import pytest

from paper_1311_2769_gb300 import serve, synth


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-5
        return self.t


class FakeExecutor:
    """Finishes a batch `service` seconds (fake clock) after submission."""

    def __init__(self, clock, slots=2, bytes_per_event=100, service=2e-3):
        self.clock, self.slots, self.bytes_per_event, self.service = clock, slots, bytes_per_event, service
        self.running = {}
        self.peak_concurrency = 0

    def submit(self, slot, events):
        assert slot not in self.running
        self.running[slot] = (self.clock() + self.service, events)
        self.peak_concurrency = max(self.peak_concurrency, len(self.running))

    def poll(self, slot):
        t_end, evs = self.running[slot]
        if self.clock() < t_end:
            return None
        del self.running[slot]
        return [serve.EventResult(e.eid, 0, 0) for e in evs]


def _events(n, rate, seed=0):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    z = np.zeros(3, np.float32)
    return [serve.Event(i, float(t[i]), z, z, z.astype(np.int8)) for i in range(n)]


def test_scheduler_respects_memory_budget_and_batch_size():
    clk = FakeClock()
    ex = FakeExecutor(clk, slots=3, bytes_per_event=100, service=5e-3)
    sch = serve.Scheduler(ex, budget_bytes=100 * 40, max_batch=16, clock=clk)
    evs = _events(500, rate=20000)
    done = sch.run(evs, t0=0.0)
    assert sorted(done) == list(range(500))
    assert sch.max_inflight_bytes <= 100 * 40
    assert max(n for _, n, _ in sch.batches) <= 16
    assert ex.peak_concurrency >= 2          # batches overlap (continuous batching)
    # every event completes after it arrives, and FIFO admission keeps order per slot wave
    for e in evs:
        assert done[e.eid][1] >= e.arrival
    st = serve.latency_stats(evs, done)
    assert st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_scheduler_rejects_event_larger_than_budget():
    clk = FakeClock()
    with pytest.raises(ValueError):
        serve.Scheduler(FakeExecutor(clk, bytes_per_event=1000), budget_bytes=999, max_batch=4, clock=clk)


def test_admission_waits_for_memory():
    clk = FakeClock()
    ex = FakeExecutor(clk, slots=4, bytes_per_event=100, service=1e-3)
    sch = serve.Scheduler(ex, budget_bytes=250, max_batch=8, clock=clk)
    evs = _events(50, rate=1e6)
    done = sch.run(evs, t0=0.0)
    assert len(done) == 50 and sch.max_inflight_bytes <= 250
    assert max(n for _, n, _ in sch.batches) <= 2


@pytest.mark.gpu
def test_result_same_alone_and_in_the_mix(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_2769_gb300 import build, ht
    build.build()
    w = synth.WORKLOADS["serving_lognormal"]
    evs = serve.poisson_trace(50000.0, 400, seed=4)
    rng = np.random.default_rng(0)
    sample = set(int(v) for v in rng.choice(400, 12, replace=False))
    kept = {}

    def consumer(eid, peaks, offsets, hits, hit_base):
        if eid in sample:
            kept[eid] = (peaks[:, 1:].copy(), (offsets - offsets[0]).copy(), (hits - hit_base).copy())

    ex = serve.GpuExecutor(w.grid, w.spec.layers, w.threshold, w.window, slots=3, max_batch=64,
                           max_hits=1 << 21, peak_cap=1 << 22, pair_cap=1 << 27, consumer=consumer)
    sch = serve.Scheduler(ex, 40 << 30, 64)
    done = sch.run(evs)
    ex.close()
    assert len(done) == 400 and len(sch.batches) > 3 and set(kept) == sample
    # alone: each sampled event in a batch of its own
    for eid in sorted(sample):
        e = evs[eid]
        ctx = ht.Context(w.grid, w.spec.layers)
        b = synth.from_arrays(e.x, e.y, layer=e.layer)
        res = ht.Results(1 << 20, 1 << 25, device="cuda")
        ctx.process(ht.Hits.from_batch(b, device="cuda"), w.threshold, w.window, res)
        ctx.sync()
        pk, po, hi = res.host()
        ctx.close()
        peaks, offsets, hits = kept[eid]
        want = np.stack([pk["i_phi"], pk["i_d0"], pk["i_kappa"], pk["votes"].astype(np.int32)], 1)
        assert np.array_equal(peaks, want)
        assert np.array_equal(offsets, po) and np.array_equal(hits, hi)
        assert done[eid][0].n_peaks == len(pk) and done[eid][0].n_pairs == len(hi)
    # the served results against the oracle (events of at most 6000 hits
    # keep the single-threaded oracle quick)
    checked = 0
    for eid in sorted(sample):
        e = evs[eid]
        if len(e.x) > 6000:
            continue
        acc = oracle_mod.vote(w.grid, e.x, e.y)
        opk = oracle_mod.peaks(w.grid, acc, w.threshold)
        opo, ohi = oracle_mod.associate(w.grid, e.x, e.y, None, opk, w.window)
        peaks, offsets, hits = kept[eid]
        want = np.stack([opk["i_phi"], opk["i_d0"], opk["i_kappa"], opk["votes"].astype(np.int32)], 1)
        assert np.array_equal(peaks, want)
        assert np.array_equal(offsets, opo) and np.array_equal(hits, ohi)
        checked += 1
    assert checked >= 6
