"""The association through the per-layer angular index (HT_OPT_ASSOC_INDEX,
the default) gives the same rows as binning every hit in every column, on
every workload shape: batch events, the dense event with displaced tracks,
windows 0..3, small and ragged grids, and the 80k-hit pileup events (buckets
sorted in global memory, events wider than one bitmap segment)."""

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_2769_gb300 import build, ht as mod
    build.build()
    mod.load()
    return mod


def _both(ht, g, b, thr, window, peak_cap=1 << 22, pair_cap=1 << 28):
    out = []
    hits = ht.Hits.from_batch(b, device="cuda")
    for use in (0, 1):
        ctx = ht.Context(g, b.layer_r)
        ctx.set_option(ht.HT_OPT_ASSOC_INDEX, use)
        assert ctx.get_option(ht.HT_OPT_ASSOC_INDEX) == use
        res = ht.Results(peak_cap, pair_cap, device="cuda")
        ctx.process(hits, thr, window, res)
        ctx.sync()
        out.append(res.host())
        ctx.close()
    (pk0, po0, hi0), (pk1, po1, hi1) = out
    assert np.array_equal(pk0, pk1) and np.array_equal(po0, po1)
    assert np.array_equal(hi0, hi1)
    return pk1, po1, hi1


@pytest.mark.parametrize("window", [0, 1, 3])
def test_index_equals_scan_batch(ht, window):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=64, first_event=100)
    pk, po, hi = _both(ht, w.grid, b, w.threshold, window)
    assert len(hi) > 100000


def test_index_equals_scan_dense_and_single(ht, oracle_mod):
    w = synth.WORKLOADS["dense_event_500trk"]
    b = synth.generate(w)
    _both(ht, w.grid, b, w.threshold, 1)
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w, n_events=5)
    pk, po, hi = _both(ht, w.grid, b, 3, 2)
    po_o, hi_o = oracle_mod.associate(w.grid, b.x, b.y, b.event_offsets, pk, 2)
    assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o)


def test_index_equals_scan_ragged_grid(ht, oracle_mod):
    g = synth.Grid(37, 13, 45, -31.0, 23.0, -0.011, 0.0137)
    b = synth.generate(synth.WORKLOADS["batch_4096_lognormal"], n_events=6, first_event=3)
    pk, po, hi = _both(ht, g, b, 7, 1)
    acc = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc, 7)
    po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o, 1)
    assert np.array_equal(pk, pk_o) and np.array_equal(po, po_o) and np.array_equal(hi, hi_o)


def test_index_equals_scan_pileup(ht):
    w = synth.WORKLOADS["pileup_64x5000trk"]
    b = synth.generate(w, n_events=2)
    assert np.diff(b.event_offsets).max() > 16384  # several bitmap segments per event
    _both(ht, w.grid, b, w.threshold, 1, peak_cap=1 << 23, pair_cap=1 << 30)


def test_index_with_pair_cap_cut(ht):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=8, first_event=30)
    pk, po, hi = _both(ht, w.grid, b, w.threshold, 1)
    qc = int(po[len(pk) // 2]) + 7
    hits = ht.Hits.from_batch(b, device="cuda")
    got = []
    for use in (0, 1):
        ctx = ht.Context(w.grid, b.layer_r)
        ctx.set_option(ht.HT_OPT_ASSOC_INDEX, use)
        res = ht.Results(1 << 22, qc, device="cuda")
        ctx.process(hits, w.threshold, 1, res)
        with pytest.raises(ht.HtError) as ei:
            ctx.sync()
        assert ei.value.status == ht.HT_ERR_OVERFLOW
        got.append(res.hit_idx[:qc].cpu().numpy())
        ctx.close()
    assert np.array_equal(got[0], got[1]) and np.array_equal(got[1], hi[:qc])
