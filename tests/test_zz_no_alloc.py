"""The allocation-free peak finder agrees with ht_peaks.

Callers that cannot allocate device memory (inside a framework that owns all
allocations, on a real-time path, without a context) use ht_peaks_noalloc,
whose scratch is a fixed device array shared by every call.  This file is
collected last so a failure here leaves every other test already run; it
passes alone in a fresh process and after the others.
"""

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_peaks_match_ht_peaks_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_2769_gb300 import build, ht
    build.build()
    w = synth.WORKLOADS["batch_4096_lognormal"]
    g = w.grid
    cells = g.n_phi * g.n_d0 * g.n_kappa
    batches = [synth.generate(w, n_events=6, first_event=0), synth.generate(w, n_events=3, first_event=50)]
    cap = 1 << 20
    for b in batches:  # two calls in a row on different inputs: no state leaks between calls
        ctx = ht.Context(g, w.spec.layers)
        ctx.vote(ht.Hits.from_batch(b, device="cuda"))
        acc = np.stack([ctx.accumulator(e) for e in range(b.n_events)])
        want = ctx.peaks(w.threshold)
        ctx.close()
        acc_d = torch.from_numpy(acc.reshape(-1)).cuda()
        peaks = torch.zeros((cap, 5), dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        ht.ht_peaks_noalloc(g, acc_d, b.n_events, w.threshold, peaks, cap, count)
        torch.cuda.synchronize()
        n = int(count.item())
        got = peaks[:n].cpu().numpy().view(np.int32).reshape(-1, 5).copy().view(ht.PEAK_DTYPE).reshape(-1)
        assert n == len(want)
        assert np.array_equal(got, want)


def test_noalloc_rejects_work_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_2769_gb300 import build, ht
    build.build()
    g = synth.WORKLOADS["pileup_64x5000trk"].grid   # 131072 columns x 108 B per event
    acc = torch.zeros(1, dtype=torch.uint32 if hasattr(torch, "uint32") else torch.int32, device="cuda")
    peaks = torch.zeros((1, 5), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(ht.HtError) as ei:
        ht.ht_peaks_noalloc(g, acc, 8, 10, peaks, 1, count)
    assert ei.value.status == ht.HT_ERR_BUDGET
