"""GPU parity of range voting (HT_VOTE_RANGE) against the oracle.

Accumulators, peak lists and association CSR must equal the oracle's range
vote and range association bit for bit; the counting pass's row lengths and
the pair totals must hold under waves and output caps too.
"""

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


def _ctx(ht, grid, opts=()):
    ctx = ht.Context(grid, synth.LAYERS_13)
    ctx.set_option(ht.HT_OPT_VOTE_MODE, ht.HT_VOTE_RANGE)
    for k, v in opts:
        ctx.set_option(k, v)
    return ctx


def _run(ht, grid, batch, thr, window, opts=(), peak_cap=1 << 22, pair_cap=1 << 26, budget=None):
    ctx = _ctx(ht, grid, opts)
    if budget is not None:
        ctx.set_option(ht.HT_OPT_ACC_BUDGET, budget)
    hits = ht.Hits.from_batch(batch, device="cuda")
    res = ht.Results(peak_cap, pair_cap, device="cuda")
    ctx.process(hits, thr, window, res)
    ctx.sync()
    out = res.host()
    ctx.close()
    return out


GRIDS = [
    synth.Grid(64, 8, 64, -10.0, 10.0, -0.0114, 0.0114),      # the single-event grid
    synth.Grid(37, 13, 45, -21.0, 17.0, -0.013, 0.009),       # ragged, asymmetric kappa range
    synth.Grid(16, 4, 512, -10.0, 10.0, -0.0114, 0.0114),     # wide kappa axis
    synth.Grid(40, 9, 32, -10.0, 10.0, 0.001, 0.02),          # kappa range not containing 0
]


@pytest.mark.parametrize("gi", range(len(GRIDS)))
def test_range_vote_equals_oracle(ht, oracle_mod, gi):
    g = GRIDS[gi]
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w, n_events=3)
    ctx = _ctx(ht, g)
    ctx.vote(ht.Hits.from_batch(b, device="cuda"))
    acc_o = oracle_mod.vote_range(g, b.x, b.y, b.event_offsets)
    for e in range(b.n_events):
        assert np.array_equal(ctx.accumulator(e), acc_o[e]), (gi, e)
    ctx.close()


def test_range_vote_tiles_and_threads(ht, oracle_mod):
    g = synth.Grid(48, 12, 64, -25.0, 25.0, -0.0114, 0.0114)
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=2, first_event=40)
    acc_o = oracle_mod.vote_range(g, b.x, b.y, b.event_offsets)
    for tp, td, thr in ((1, 12, 256), (2, 5, 128), (4, 12, 256), (8, 3, 256)):
        ctx = _ctx(ht, g, ((ht.HT_OPT_TILE_PHI, tp), (ht.HT_OPT_TILE_D0, td), (ht.HT_OPT_THREADS, thr)))
        ctx.vote(ht.Hits.from_batch(b, device="cuda"))
        for e in range(b.n_events):
            assert np.array_equal(ctx.accumulator(e), acc_o[e]), (tp, td, thr, e)
        ctx.close()


@pytest.mark.parametrize("window", [0, 1, 2])
def test_range_process_equals_oracle(ht, oracle_mod, window):
    """Peaks and the full association CSR of range voting, on three events of
    the single-event workload and two events of the batch workload."""
    for wname, n, thr in (("single_event_10trk", 3, 8), ("batch_4096_lognormal", 2, 12)):
        w = synth.WORKLOADS[wname]
        g = w.grid if wname == "single_event_10trk" else synth.Grid(64, 16, 64, -25.0, 25.0, -0.0114, 0.0114)
        b = synth.generate(w, n_events=n, first_event=11)
        acc_o = oracle_mod.vote_range(g, b.x, b.y, b.event_offsets)
        pk_o = oracle_mod.peaks(g, acc_o, thr)
        po_o, hi_o = oracle_mod.associate_range(g, b.x, b.y, b.event_offsets, pk_o, window)
        pk, po, hi = _run(ht, g, b, thr, window)
        assert np.array_equal(pk, pk_o), wname
        assert np.array_equal(po, po_o), wname
        assert np.array_equal(hi, hi_o), wname


def test_range_association_passes_and_waves(ht, oracle_mod):
    """Row cursors walked in passes (64 cursors per warp against ~500 peaks
    per row, counting and writing) and an accumulator budget of two events
    (waves): the same CSR as the oracle's."""
    w = synth.WORKLOADS["dense_event_500trk"]
    b = synth.generate(w, n_events=1)
    sel = np.arange(0, b.n_hits, 3)
    b = synth.from_arrays(b.x[sel], b.y[sel])
    g = synth.Grid(8, 32, 512, -25.0, 25.0, -0.0114, 0.0114)
    acc_o = oracle_mod.vote_range(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 2)
    assert np.bincount(pk_o["i_phi"]).max() > 4 * 64
    po_o, hi_o = oracle_mod.associate_range(g, b.x, b.y, b.event_offsets, pk_o, 1)
    pk, po, hi = _run(ht, g, b, 2, 1, opts=((ht.HT_OPT_ASSOC_CURSORS, 64),), pair_cap=1 << 28)
    assert np.array_equal(pk, pk_o) and np.array_equal(po, po_o) and np.array_equal(hi, hi_o)
    w2 = synth.WORKLOADS["single_event_10trk"]
    b2 = synth.generate(w2, n_events=5, first_event=20)
    g2 = w2.grid
    cells = g2.n_phi * g2.n_d0 * g2.n_kappa
    one = _run(ht, g2, b2, 8, 1)
    waves = _run(ht, g2, b2, 8, 1, budget=2 * cells * 4)
    for a, c in zip(one, waves):
        assert np.array_equal(a, c)


def test_range_overflow_keeps_prefix_and_counts(ht, oracle_mod):
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w, n_events=4, first_event=2)
    g = w.grid
    full = _run(ht, g, b, 8, 1)
    ctx = _ctx(ht, g)
    pc, qc = len(full[0]) // 3, len(full[2]) // 4
    res = ht.Results(pc, qc, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), 8, 1, res)
    with pytest.raises(ht.HtError) as ei:
        ctx.sync()
    assert ei.value.status == ht.HT_ERR_OVERFLOW
    cnt = res.counts.cpu().numpy()
    assert cnt[0] == len(full[0]) and cnt[1] == len(full[2])
    pk, po, hi = res.host()
    assert np.array_equal(pk, full[0][:pc])
    m = min(qc, int(full[1][pc]))
    assert np.array_equal(hi[:m], full[2][:m])
    ctx.close()


def test_range_host_calls(ht, oracle_mod):
    """ht_vote / ht_peaks / ht_associate in range mode, host outputs."""
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w, n_events=2, first_event=30)
    g = w.grid
    ctx = _ctx(ht, g)
    ctx.vote(ht.Hits.from_batch(b))
    pk = ctx.peaks(8)
    acc_o = oracle_mod.vote_range(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 8)
    assert np.array_equal(pk, pk_o)
    po, hi = ctx.associate(1, len(pk))
    po_o, hi_o = oracle_mod.associate_range(g, b.x, b.y, b.event_offsets, pk_o, 1)
    assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o)
    assert ctx.get_option(ht.HT_OPT_VOTE_MODE) == ht.HT_VOTE_RANGE
    ctx.close()
