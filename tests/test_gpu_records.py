"""Association over the vote's records against binning every cell again and
against the oracle (Section 3: a hit joins a maximum it voted near).

The band vote writes, per (hit, tile) whose d0 band meets the tile, the
tile's bins; the association reads them.  Every case compares the records
path with the binning path (HT_OPT_RECORDS 0) element by element, and rows
with the oracle: record sizes of 32, 64, 128 and 256 cells (1, 2, 4 and 8
cells per lane), ragged tiles at the phi and d0 edges, windows 0 to 6,
waves split by the record budget (host and device hits, including read-back
offsets), an event whose records alone exceed the budget, cursor passes and
output caps.
"""

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_2769_gb300 import build, ht as mod
    build.build()
    mod.load()
    return mod


def _run(ht, grid, batch, thr, window, records, opts=(), device_io=True, peak_cap=1 << 22, pair_cap=1 << 27,
         expect_records=None):
    ctx = ht.Context(grid, synth.LAYERS_13)
    ctx.set_option(ht.HT_OPT_RECORDS, records)
    for k, v in opts:
        ctx.set_option(k, v)
    if expect_records is not None:
        assert ctx.get_option(ht.HT_OPT_RECORDS) == expect_records
    hits = ht.Hits.from_batch(batch, device="cuda" if device_io else None)
    res = ht.Results(peak_cap, pair_cap, device="cuda" if device_io else None)
    ctx.process(hits, thr, window, res)
    ctx.sync()
    out = res.host()
    ctx.close()
    return out


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def _rows_vs_oracle(oracle_mod, grid, batch, pk, po, hi, window, sample=400, seed=0):
    if len(pk) == 0:
        return
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(pk), min(sample, len(pk)), replace=False))
    po_o, hi_o = oracle_mod.associate(grid, batch.x, batch.y, batch.event_offsets, pk[sel], window)
    for t, p in enumerate(sel):
        assert np.array_equal(hi[po[p]:po[p + 1]], hi_o[po_o[t]:po_o[t + 1]]), (p, pk[p])


@pytest.fixture(scope="module")
def batch5():
    w = synth.WORKLOADS["batch_4096_lognormal"]
    return synth.generate(w, n_events=5, first_event=40)


@pytest.mark.parametrize("tile", [(1, 32, 128), (2, 16, 256), (4, 16, 128), (4, 32, 128), (8, 32, 256),
                                  (8, 4, 256)])
def test_record_tiles_equal_binning_and_oracle(ht, oracle_mod, batch5, tile):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    opts = ((ht.HT_OPT_TILE_PHI, tile[0]), (ht.HT_OPT_TILE_D0, tile[1]), (ht.HT_OPT_THREADS, tile[2]))
    rec = _run(ht, w.grid, batch5, w.threshold, w.window, 1, opts, expect_records=1)
    ref = _run(ht, w.grid, batch5, w.threshold, w.window, 0, opts, expect_records=0)
    _same(rec, ref)
    assert len(rec[2]) > 100000
    _rows_vs_oracle(oracle_mod, w.grid, batch5, *rec, w.window, sample=300, seed=tile[0] * 100 + tile[1])


def test_records_ragged_grid_full_oracle(ht, oracle_mod):
    """50 phi rows in tiles of 4 (two rows left over) and 20 d0 columns in
    tiles of 16 (four left over): the tile's missing cells hold no peaks."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=3, first_event=7)
    g = synth.Grid(50, 20, 40, -25.0, 25.0, -0.0114, 0.0114)
    opts = ((ht.HT_OPT_TILE_PHI, 4), (ht.HT_OPT_TILE_D0, 16))
    pk, po, hi = _run(ht, g, b, 5, 1, 1, opts, expect_records=1)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 5)
    assert np.array_equal(pk, pk_o)
    po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o, 1)
    assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o)


@pytest.mark.parametrize("window", [0, 1, 2, 3, 6])
def test_records_windows_full_oracle(ht, oracle_mod, window):
    """A low threshold on a dense event: bins whose window holds two or more
    peaks of a column."""
    w = synth.WORKLOADS["dense_event_500trk"]
    b = synth.generate(w, n_events=1)
    g = synth.Grid(48, 16, 64, -25.0, 25.0, -0.0114, 0.0114)
    opts = ((ht.HT_OPT_TILE_PHI, 4), (ht.HT_OPT_TILE_D0, 16))
    pk, po, hi = _run(ht, g, b, 3, window, 1, opts, expect_records=1)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 3)
    assert np.array_equal(pk, pk_o)
    po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o, window)
    assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o)


@pytest.mark.parametrize("device_io", [True, False])
def test_record_budget_splits_waves(ht, oracle_mod, device_io):
    """A record budget of about a third of the batch's records: waves by
    record memory (device hits: offsets read back), same results; a budget
    below one event's records: that call bins again, same results."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=24, first_event=100)
    g = w.grid
    opts = ((ht.HT_OPT_TILE_PHI, 4), (ht.HT_OPT_TILE_D0, 16), (ht.HT_OPT_THREADS, 128))
    one = _run(ht, g, b, w.threshold, w.window, 1, opts, device_io=device_io)
    per_hit = g.n_phi * g.n_d0  # record bytes per hit: one per cell of every tile
    budget = b.n_hits * per_hit // 3
    split = _run(ht, g, b, w.threshold, w.window, 1, opts + ((ht.HT_OPT_RECORD_BUDGET, budget),),
                 device_io=device_io)
    _same(one, split)
    small = int(np.diff(b.event_offsets).max()) * per_hit - 1
    fallback = _run(ht, g, b, w.threshold, w.window, 1, opts + ((ht.HT_OPT_RECORD_BUDGET, small),),
                    device_io=device_io)
    _same(one, fallback)
    _rows_vs_oracle(oracle_mod, g, b, *split, w.window, sample=300, seed=5)


def test_record_waves_with_accumulator_budget_and_plain_mode(ht, oracle_mod):
    """Waves from the accumulator budget and from the record budget at once,
    and the plain one-event-per-launch form, all equal."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=9, first_event=500)
    g = w.grid
    cells = g.n_phi * g.n_d0 * g.n_kappa
    base = _run(ht, g, b, w.threshold, w.window, 0)
    both = _run(ht, g, b, w.threshold, w.window, 1,
                ((ht.HT_OPT_ACC_BUDGET, 4 * cells * 4), (ht.HT_OPT_RECORD_BUDGET, b.n_hits * g.n_phi * g.n_d0 // 2)))
    _same(base, both)
    plain = _run(ht, g, b, w.threshold, w.window, 1, ((ht.HT_OPT_MODE, ht.HT_MODE_PLAIN),))
    _same(base, plain)


def test_record_cursor_passes(ht, oracle_mod, batch5):
    """32 row cursors per warp against ~100 peaks per tile: every tile is
    walked in several passes over its records."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    opts = ((ht.HT_OPT_TILE_PHI, 4), (ht.HT_OPT_TILE_D0, 16))
    full = _run(ht, w.grid, batch5, w.threshold, 1, 1, opts)
    small = _run(ht, w.grid, batch5, w.threshold, 1, 1, opts + ((ht.HT_OPT_ASSOC_CURSORS, 32),))
    _same(full, small)


def test_record_output_caps(ht):
    """Peak and pair caps with records: the stored prefix and the true counts
    of an unbounded run, across record waves."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=6, first_event=300)
    g = synth.Grid(64, 16, 32, -25.0, 25.0, -0.0114, 0.0114)
    opts = ((ht.HT_OPT_RECORD_BUDGET, b.n_hits * g.n_phi * g.n_d0 // 3),)
    full = _run(ht, g, b, 5, 1, 1, opts)
    for pc, qc in ((50, 400), (len(full[0]) // 3, len(full[2]) // 4)):
        ctx = ht.Context(g, w.spec.layers)
        for k, v in opts:
            ctx.set_option(k, v)
        res = ht.Results(pc, qc, device="cuda")
        ctx.process(ht.Hits.from_batch(b, device="cuda"), 5, 1, res)
        with pytest.raises(ht.HtError) as ei:
            ctx.sync()
        assert ei.value.status == ht.HT_ERR_OVERFLOW
        cnt = res.counts.cpu().numpy()
        assert cnt[0] == len(full[0]) and cnt[1] == len(full[2])
        pk, po, hi = res.host()
        assert np.array_equal(pk, full[0][:pc])
        m = min(qc, int(full[1][len(pk)]))
        assert np.array_equal(hi[:m], full[2][:m])
        ctx.close()


def test_records_unsupported_shapes_bin_again(ht):
    """A 256-bin kappa axis (bins need more than a byte) and a 96-cell tile
    keep the binning association."""
    g = synth.Grid(32, 16, 256, -25.0, 25.0, -0.0114, 0.0114)
    ctx = ht.Context(g, synth.LAYERS_13)
    assert ctx.get_option(ht.HT_OPT_RECORDS) == 0
    ctx.close()
    g = synth.Grid(48, 12, 64, -25.0, 25.0, -0.0114, 0.0114)
    ctx = ht.Context(g, synth.LAYERS_13)
    ctx.set_option(ht.HT_OPT_TILE_PHI, 8)
    ctx.set_option(ht.HT_OPT_TILE_D0, 12)
    assert ctx.get_option(ht.HT_OPT_RECORDS) == 0
    ctx.close()


def test_phase_timing_over_waves_and_host_chunks(ht):
    """Phase times are summed over waves, with graph replay (device results)
    and with direct launches (host results copied wave by wave)."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=12, first_event=900)
    g = w.grid
    for device_io in (True, False):
        ctx = ht.Context(g, synth.LAYERS_13)
        ctx.set_option(ht.HT_OPT_PHASE_TIMING, 1)
        ctx.set_option(ht.HT_OPT_RECORD_BUDGET, b.n_hits * g.n_phi * g.n_d0 // 3)
        hits = ht.Hits.from_batch(b, device="cuda" if device_io else None)
        res = ht.Results(1 << 22, 1 << 27, device="cuda" if device_io else None)
        for _ in range(2):
            ctx.process(hits, w.threshold, w.window, res)
            ctx.sync()
        assert ctx.get_option(ht.HT_OPT_WAVES) >= 3
        v, r, total, a = ctx.phase_times()
        assert v > 0 and r > 0 and 0 < a <= r and v + r <= total * 1.05
        ctx.close()


def test_closing_a_context_frees_its_records(ht):
    """A context's device memory, records included, is returned on close."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=64, first_event=1000)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ctx = ht.Context(w.grid, synth.LAYERS_13)
    res = ht.Results(1 << 22, 1 << 26, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), w.threshold, w.window, res)
    ctx.sync()
    assert ctx.get_option(ht.HT_OPT_RECORDS) == 1
    free1, _ = torch.cuda.mem_get_info()
    held = free0 - free1
    assert held > b.n_hits * w.grid.n_phi * w.grid.n_d0  # the records at least
    ctx.close()
    del res
    torch.cuda.empty_cache()
    free2, _ = torch.cuda.mem_get_info()
    assert free0 - free2 < 64 << 20, (free0 - free2) / 2 ** 20
