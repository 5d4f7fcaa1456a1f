"""The allocation-free peak finder agrees with ht_peaks and with the oracle.

Callers that cannot allocate device memory where they need peaks (code inside
a framework that owns every device allocation, a real-time path that must not
block on cudaMalloc, code without a context object) use ht_peaks_noalloc,
whose scratch is a fixed device array shared by every call.  This file is
collected last so a failure here leaves every other test already run; it
passes alone in a fresh process and after the others.  Every call goes
through the C ABI (the binding's checks only guard argument shapes).
"""

import ctypes

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_2769_gb300 import build, ht
    build.build()
    return ht


def _acc_of(ht, w, b):
    ctx = ht.Context(w.grid, w.spec.layers)
    ctx.vote(ht.Hits.from_batch(b, device="cuda"))
    acc = np.stack([ctx.accumulator(e) for e in range(b.n_events)])
    want = ctx.peaks(w.threshold)
    ctx.close()
    return acc, want


def _noalloc(ht, g, acc_d, n_events, thr, cap, stream=None):
    peaks = torch.zeros((max(cap, 1), 5), dtype=torch.int32, device="cuda")
    count = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    ht.ht_peaks_noalloc(g, acc_d, n_events, thr, peaks, cap, count, stream=stream)
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    n = int(count.item())
    got = peaks[:min(n, cap)].cpu().numpy().view(np.int32).reshape(-1, 5).copy().view(ht.PEAK_DTYPE).reshape(-1)
    return n, got


def test_noalloc_peaks_match_ht_peaks_and_oracle_twice_in_a_row(oracle_mod):
    ht = _need_gpu()
    w = synth.WORKLOADS["batch_4096_lognormal"]
    g = w.grid
    batches = [synth.generate(w, n_events=6, first_event=0), synth.generate(w, n_events=3, first_event=50)]
    cap = 1 << 20
    for b in batches:  # two calls in a row on different inputs: no state leaks between calls
        acc, want = _acc_of(ht, w, b)
        acc_d = torch.from_numpy(acc.reshape(-1).view(np.int32)).cuda()
        n, got = _noalloc(ht, g, acc_d, b.n_events, w.threshold, cap)
        assert n == len(want)
        assert np.array_equal(got, want)
        # the oracle's peaks of the same accumulators (the accumulators
        # themselves are bit-exact against the oracle in the parity tests)
        assert np.array_equal(got, oracle_mod.peaks(g, acc, w.threshold))


def test_noalloc_cap_empty_stream_and_odd_kappa(oracle_mod):
    ht = _need_gpu()
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=2, first_event=7)
    acc, want = _acc_of(ht, w, b)
    acc_d = torch.from_numpy(acc.reshape(-1).view(np.int32)).cuda()
    # cap 1: the count is still the true total and the first peak is right
    n, got = _noalloc(ht, w.grid, acc_d, b.n_events, w.threshold, 1)
    assert n == len(want) and len(got) == 1 and got[0] == want[0]
    # no events: count 0
    n, got = _noalloc(ht, w.grid, acc_d, 0, w.threshold, 16)
    assert n == 0
    # an explicit non-default stream
    s = torch.cuda.Stream()
    n, got = _noalloc(ht, w.grid, acc_d, b.n_events, w.threshold, 1 << 20, stream=s)
    assert n == len(want) and np.array_equal(got, want)
    # n_kappa not a multiple of 4 (scalar row loads), against the oracle
    g = synth.Grid(24, 6, 30, -25.0, 25.0, -0.0114, 0.0114)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    acc_d = torch.from_numpy(acc_o.reshape(-1).view(np.int32)).cuda()
    n, got = _noalloc(ht, g, acc_d, b.n_events, 6, 1 << 16)
    want_o = oracle_mod.peaks(g, acc_o, 6)
    assert n == len(want_o) and n > 0 and np.array_equal(got, want_o)


def test_noalloc_does_not_lower_a_context_shared_memory_limit():
    """A context on the single-event grid (its detection tile needs more
    shared memory) keeps working after an allocation-free call on the batch
    grid (a smaller tile)."""
    ht = _need_gpu()
    w1 = synth.WORKLOADS["single_event_10trk"]
    b1 = synth.generate(w1)
    ctx = ht.Context(w1.grid, w1.spec.layers)
    ctx.vote(ht.Hits.from_batch(b1, device="cuda"))
    want = ctx.peaks(w1.threshold)
    w = synth.WORKLOADS["batch_4096_lognormal"]
    acc, _ = _acc_of(ht, w, synth.generate(w, n_events=1))
    acc_d = torch.from_numpy(acc.reshape(-1).view(np.int32)).cuda()
    _noalloc(ht, w.grid, acc_d, 1, w.threshold, 1 << 16)
    assert np.array_equal(ctx.peaks(w1.threshold), want)
    ctx.close()


def _raw_call(ht, g, acc_ptr, n_events, peaks_ptr, cap, count_ptr):
    gs = ht.HtGrid(g.n_phi, g.n_d0, g.n_kappa, g.d0_min, g.d0_max, g.kappa_min, g.kappa_max)
    return ht.load().ht_peaks_noalloc(ctypes.byref(gs), acc_ptr, int(n_events), 9, peaks_ptr, int(cap), count_ptr,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_budget_boundary_and_bad_pointers():
    ht = _need_gpu()
    g = synth.WORKLOADS["batch_4096_lognormal"].grid  # 8192 columns x 36 B per event: 113 events fit in 32 MiB
    cells = g.n_phi * g.n_d0 * g.n_kappa
    acc = torch.zeros(114 * cells, dtype=torch.int32, device="cuda")
    peaks = torch.zeros((16, 5), dtype=torch.int32, device="cuda")
    count = torch.zeros(2, dtype=torch.int64, device="cuda")
    assert _raw_call(ht, g, acc.data_ptr(), 113, peaks.data_ptr(), 16, count.data_ptr()) == ht.HT_OK
    torch.cuda.synchronize()
    assert int(count[0].item()) == 0
    assert _raw_call(ht, g, acc.data_ptr(), 114, peaks.data_ptr(), 16, count.data_ptr()) == ht.HT_ERR_BUDGET
    # a huge event count is refused before any size arithmetic could wrap
    assert _raw_call(ht, g, acc.data_ptr(), 2**31 - 1, peaks.data_ptr(), 16, count.data_ptr()) == ht.HT_ERR_BUDGET
    # misaligned accumulators (16-byte row loads), count and peaks
    assert _raw_call(ht, g, acc.data_ptr() + 4, 1, peaks.data_ptr(), 16, count.data_ptr()) == ht.HT_ERR_INVALID_ARG
    assert _raw_call(ht, g, acc.data_ptr(), 1, peaks.data_ptr(), 16, count.data_ptr() + 4) == ht.HT_ERR_INVALID_ARG
    assert _raw_call(ht, g, acc.data_ptr(), 1, peaks.data_ptr() + 2, 16, count.data_ptr()) == ht.HT_ERR_INVALID_ARG
    torch.cuda.synchronize()
    # the binding refuses tensors too small for the call
    with pytest.raises(ValueError):
        ht.ht_peaks_noalloc(g, acc[:10], 1, 9, peaks, 16, count[:1])
    with pytest.raises(ValueError):
        ht.ht_peaks_noalloc(g, acc, 1, 9, peaks, 17, count[:1])


def test_noalloc_rejects_work_beyond_its_scratch():
    ht = _need_gpu()
    g = synth.WORKLOADS["pileup_64x5000trk"].grid   # 131072 columns x 108 B per event
    acc = torch.zeros(4, dtype=torch.int32, device="cuda")
    peaks = torch.zeros((1, 5), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert _raw_call(ht, g, acc.data_ptr(), 8, peaks.data_ptr(), 1, count.data_ptr()) == ht.HT_ERR_BUDGET
