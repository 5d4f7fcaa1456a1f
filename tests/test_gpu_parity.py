"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Accumulators, peak lists and association CSR must be bit-exact.  Small
workloads are compared in full; the full-size batch (4096 ragged events,
the benchmarked launch configuration) and the 80k-hit pileup events are
compared on sampled events, columns and peaks.
"""

import math

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


def _run(ht, grid, batch, thr, window, device_io=True, mode=None, budget=None, opts=(), peak_cap=1 << 22,
         pair_cap=1 << 26, layer_r=synth.LAYERS_13):
    ctx = ht.Context(grid, layer_r)
    if mode is not None:
        ctx.set_option(ht.HT_OPT_MODE, mode)
    if budget is not None:
        ctx.set_option(ht.HT_OPT_ACC_BUDGET, budget)
    for k, v in opts:
        ctx.set_option(k, v)
    hits = ht.Hits.from_batch(batch, device="cuda" if device_io else None)
    res = ht.Results(peak_cap, pair_cap, device="cuda" if device_io else None)
    ctx.process(hits, thr, window, res)
    ctx.sync()
    out = res.host()
    ctx.close()
    return out


def _check_csr_rows(oracle_mod, grid, batch, pk, po, hi, window, sample, seed=0):
    """Association rows of sampled peaks against the oracle."""
    if len(pk) == 0:
        return
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(pk), min(sample, len(pk)), replace=False))
    po_o, hi_o = oracle_mod.associate(grid, batch.x, batch.y, batch.event_offsets, pk[sel], window)
    for t, p in enumerate(sel):
        assert np.array_equal(hi[po[p]:po[p + 1]], hi_o[po_o[t]:po_o[t + 1]]), f"peak {p} {pk[p]}"


# ---------------------------------------------------------------- primitives

def test_rcp_approx_error_bound(ht):
    """The stage-1 bound assumes |rcp(x) x - 1| <= 2^-22 for positive normals."""
    for first in (0x3F800000, 0x3A800000, 0x4B000000, 0x00800000 + (1 << 23) * 3):
        worst, n = ht.ht_check_rcp(first, 1 << 23)
        assert n == 1 << 23
        assert worst <= (1 << 18), (hex(first), worst / 2 ** 40)


def test_tables_match_oracle(ht, oracle_mod):
    for w in synth.WORKLOADS.values():
        ctx = ht.Context(w.grid, w.spec.layers)
        c, s, d = ctx.tables()
        co, so, do = oracle_mod.tables(w.grid)
        assert np.array_equal(c, co) and np.array_equal(s, so) and np.array_equal(d, do)
        ctx.close()


# ---------------------------------------------------------------- whole small workloads

@pytest.mark.parametrize("device_io", [True, False])
def test_single_event_full_parity(ht, oracle_mod, device_io):
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w)
    ctx = ht.Context(w.grid, w.spec.layers)
    ctx.vote(ht.Hits.from_batch(b, device="cuda" if device_io else None))
    acc_o = oracle_mod.vote(w.grid, b.x, b.y, b.event_offsets)
    assert np.array_equal(ctx.accumulator(0), acc_o[0])
    for thr in (w.threshold, 4, 2):
        pk_o = oracle_mod.peaks(w.grid, acc_o, thr)
        pk = ctx.peaks(thr)
        assert np.array_equal(pk, pk_o)
        po, hi = ctx.associate(1, len(pk))
        po_o, hi_o = oracle_mod.associate(w.grid, b.x, b.y, b.event_offsets, pk_o, 1)
        assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o)
    ctx.close()


def test_dense_event_full_accumulator_and_peaks(ht, oracle_mod):
    w = synth.WORKLOADS["dense_event_500trk"]
    b = synth.generate(w)
    ctx = ht.Context(w.grid, w.spec.layers)
    ctx.vote(ht.Hits.from_batch(b, device="cuda"))
    acc_o = oracle_mod.vote(w.grid, b.x, b.y)
    assert np.array_equal(ctx.accumulator(0), acc_o[0])
    ctx.close()
    pk_o = oracle_mod.peaks(w.grid, acc_o, w.threshold)
    pk, po, hi = _run(ht, w.grid, b, w.threshold, w.window)
    assert np.array_equal(pk, pk_o)
    # every CSR row length equals the window sum of the oracle accumulator
    a = acc_o[0].astype(np.int64)
    k = pk["i_kappa"]
    win = sum(np.where((k + o >= 0) & (k + o < w.grid.n_kappa),
                       a[pk["i_phi"], pk["i_d0"], np.clip(k + o, 0, w.grid.n_kappa - 1)], 0) for o in (-1, 0, 1))
    assert np.array_equal(np.diff(po), win)
    _check_csr_rows(oracle_mod, w.grid, b, pk, po, hi, w.window, 1500)


@pytest.mark.parametrize("mode", [0, 1])
def test_modes_and_io_agree_with_oracle(ht, oracle_mod, mode):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=6, first_event=40)
    g = synth.Grid(128, 16, 64, -25.0, 25.0, -0.0114, 0.0114)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 9)
    for dev in (True, False):
        pk, po, hi = _run(ht, g, b, 9, 1, device_io=dev, mode=mode)
        assert np.array_equal(pk, pk_o)
        _check_csr_rows(oracle_mod, g, b, pk, po, hi, 1, 400)


def test_waves_equal_single_pass(ht, oracle_mod):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=9, first_event=100)
    g = synth.Grid(64, 16, 32, -25.0, 25.0, -0.0114, 0.0114)
    one = _run(ht, g, b, 9, 1)
    cells = g.n_phi * g.n_d0 * g.n_kappa
    waves = _run(ht, g, b, 9, 1, budget=2 * cells * 4)
    for a, c in zip(one, waves):
        assert np.array_equal(a, c)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    assert np.array_equal(one[0], oracle_mod.peaks(g, acc_o, 9))
    po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, one[0], 1)
    assert np.array_equal(one[1], po_o) and np.array_equal(one[2], hi_o)


def test_graph_replay_is_repeatable(ht):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=32)
    ctx = ht.Context(w.grid, w.spec.layers)
    hits = ht.Hits.from_batch(b, device="cuda")
    res = ht.Results(1 << 21, 1 << 25, device="cuda")
    outs = []
    for _ in range(3):
        ctx.process(hits, 9, 1, res)
        ctx.sync()
        outs.append(res.host())
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)
    ctx.close()


# ---------------------------------------------------------------- edge cases

def test_ragged_grid_and_explicit_tiles(ht, oracle_mod):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=2, first_event=7)
    g = synth.Grid(37, 13, 45, -21.0, 17.0, -0.013, 0.009)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 6)
    po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o, 2)
    for tp, td, thr in ((8, 5, 128), (1, 13, 256), (2, 1, 256), (4, 7, 128)):
        ctx = ht.Context(g, w.spec.layers)
        ctx.set_option(ht.HT_OPT_TILE_PHI, tp)
        ctx.set_option(ht.HT_OPT_TILE_D0, td)
        ctx.set_option(ht.HT_OPT_THREADS, thr)
        ctx.vote(ht.Hits.from_batch(b, device="cuda"))
        for e in range(2):
            assert np.array_equal(ctx.accumulator(e), acc_o[e]), (tp, td, thr, e)
        ctx.close()
        pk, po, hi = _run(ht, g, b, 6, 2, opts=((ht.HT_OPT_TILE_PHI, tp), (ht.HT_OPT_TILE_D0, td)))
        assert np.array_equal(pk, pk_o) and np.array_equal(po, po_o) and np.array_equal(hi, hi_o)


def test_empty_and_tiny_events(ht, oracle_mod):
    g = synth.Grid(16, 4, 16, -10.0, 10.0, -0.02, 0.02)
    # no events at all
    empty = synth.from_arrays(np.zeros(0), np.zeros(0), event_offsets=[0])
    pk, po, hi = _run(ht, g, empty, 1, 1)
    assert len(pk) == 0 and po.tolist() == [0] and len(hi) == 0
    # events with 0, 1 and 3 hits
    x = np.array([30.0, -12.5, 4.0, 60.0], np.float32)
    y = np.array([5.0, 40.0, -7.0, -1.0], np.float32)
    b = synth.from_arrays(x, y, event_offsets=[0, 0, 1, 1, 4])
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    ctx = ht.Context(g, synth.LAYERS_13)
    ctx.vote(ht.Hits.from_batch(b, device="cuda"))
    for e in range(4):
        assert np.array_equal(ctx.accumulator(e), acc_o[e])
    ctx.close()
    pk, po, hi = _run(ht, g, b, 1, 1)
    pk_o = oracle_mod.peaks(g, acc_o, 1)
    assert np.array_equal(pk, pk_o)
    po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o, 1)
    assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o)


def test_degenerate_hits_perigee_and_bin_edges(ht, oracle_mod):
    """Hits on perigee points (den = 0) and on bin-edge circles take the
    double-float and binary64 stages; the result must still be exact."""
    g = synth.Grid(48, 12, 64, -25.0, 25.0, -0.0114, 0.0114)
    c, s, d = oracle_mod.tables(g)
    rng = np.random.default_rng(4)
    xs, ys = [], []
    for _ in range(300):
        i, j = rng.integers(0, 48), rng.integers(0, 12)
        px, py = -float(d[j]) * float(s[i]), float(d[j]) * float(c[i])
        dist = 10.0 ** rng.uniform(-7, 0)
        a = rng.uniform(0, 2 * math.pi)
        xs.append(px + dist * math.cos(a))
        ys.append(py + dist * math.sin(a))
        xs.append(px)
        ys.append(py)
    kmin, kmax = float(np.float32(-0.0114)), float(np.float32(0.0114))
    for _ in range(300):
        i, j, k = rng.integers(0, 48), rng.integers(0, 12), rng.integers(1, 64)
        kap = kmin + k * (kmax - kmin) / 64
        hx, hy, _, ok = synth.helix_hits([math.atan2(s[i], c[i])], [float(d[j])], [kap], synth.LAYERS_13)
        xs.extend(hx[ok].tolist())
        ys.extend(hy[ok].tolist())
    b = synth.from_arrays(np.array(xs, np.float32), np.array(ys, np.float32))
    ctx = ht.Context(g, synth.LAYERS_13)
    ctx.set_option(ht.HT_OPT_COUNT_STAGES, 1)
    ctx.vote(ht.Hits.from_batch(b, device="cuda"))
    acc = ctx.accumulator(0)
    cells, st2, st3 = ctx.filter_stats()
    ctx.close()
    assert np.array_equal(acc, oracle_mod.vote(g, b.x, b.y)[0])
    assert cells == b.n_hits * 48 * 12 and st2 > 0 and st3 > 0


def test_large_kappa_axis(ht, oracle_mod):
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w)
    g = synth.Grid(8, 3, 4096, -10.0, 10.0, -0.0114, 0.0114)
    ctx = ht.Context(g, w.spec.layers)
    ctx.vote(ht.Hits.from_batch(b, device="cuda"))
    assert np.array_equal(ctx.accumulator(0), oracle_mod.vote(g, b.x, b.y)[0])
    ctx.close()


# ---------------------------------------------------------------- errors

def test_invalid_inputs_are_reported(ht):
    g = synth.Grid(16, 4, 16, -10.0, 10.0, -0.02, 0.02)
    x = np.array([1.0, np.nan, 3.0], np.float32)
    y = np.array([1.0, 2.0, 3.0], np.float32)
    for dev in (True, False):
        ctx = ht.Context(g, synth.LAYERS_13)
        b = synth.from_arrays(x, y)
        ctx.vote(ht.Hits.from_batch(b, device="cuda" if dev else None))
        with pytest.raises(ht.HtError) as ei:
            ctx.peaks(1)
        assert ei.value.status == ht.HT_ERR_INVALID_ARG
        # layer id out of range
        b2 = synth.from_arrays(y, y, layer=np.array([0, 13, 1], np.int8))
        ctx.vote(ht.Hits.from_batch(b2, device="cuda" if dev else None))
        with pytest.raises(ht.HtError):
            ctx.sync()
        ctx.close()
    ctx = ht.Context(g, synth.LAYERS_13)
    bad = synth.from_arrays(y, y, event_offsets=[0, 2, 1, 3])
    with pytest.raises(ht.HtError) as ei:
        ctx.vote(ht.Hits.from_batch(bad))
    assert ei.value.status == ht.HT_ERR_INVALID_ARG
    with pytest.raises(ht.HtError) as ei:
        ht.ht_peaks(ctx.handle, 1)
    assert ei.value.status == ht.HT_ERR_STATE
    ctx.close()


def test_overflow_and_budget(ht):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=4)
    g = synth.Grid(64, 16, 32, -25.0, 25.0, -0.0114, 0.0114)
    full = _run(ht, g, b, 5, 1)
    ctx = ht.Context(g, w.spec.layers)
    res = ht.Results(10, 100, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), 5, 1, res)
    with pytest.raises(ht.HtError) as ei:
        ctx.sync()
    assert ei.value.status == ht.HT_ERR_OVERFLOW
    cnt = res.counts.cpu().numpy()
    assert cnt[0] == len(full[0]) and cnt[1] == len(full[2])
    pk, po, hi = res.host()
    assert np.array_equal(pk, full[0][:10])
    # rows that end below the pair cap are exact; the crossing row holds its first hits
    po_full, hi_full = full[1], full[2]
    assert np.array_equal(hi[:100], hi_full[:100])
    ctx.set_option(ht.HT_OPT_ACC_BUDGET, g.n_phi * g.n_d0 * g.n_kappa * 4 * 2)
    with pytest.raises(ht.HtError) as ei:
        ctx.vote(ht.Hits.from_batch(b, device="cuda"))
    assert ei.value.status == ht.HT_ERR_BUDGET
    ctx.close()


# ---------------------------------------------------------------- full sizes, sampled

@pytest.fixture(scope="module")
def c2_batch():
    return synth.generate(synth.WORKLOADS["batch_4096_lognormal"])


def test_full_batch_sampled(ht, oracle_mod, c2_batch):
    """The benchmarked configuration: 4096 ragged events, one persistent
    launch per kernel, CUDA graph; sampled events checked in full."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = c2_batch
    nh = np.diff(b.event_offsets)
    sample = sorted({int(np.argmax(nh)), int(np.argmin(nh)), 0, 4095, 1234, 2047})
    ctx = ht.Context(w.grid, w.spec.layers)
    hits = ht.Hits.from_batch(b, device="cuda")
    res = ht.Results(1 << 27, 3 << 30, device="cuda")
    ctx.process(hits, w.threshold, w.window, res)
    ctx.sync()
    cnt = res.counts.cpu().numpy()
    ev = res.peaks[: int(cnt[0]), 0].cpu().numpy()
    assert np.all(np.diff(ev) >= 0)
    po_all = res.peak_offsets[: int(cnt[0]) + 1].cpu().numpy()
    assert po_all[-1] == cnt[1]
    for e in sample:
        be = b.event(e)
        acc_o = oracle_mod.vote(w.grid, be.x, be.y)
        pk_o = oracle_mod.peaks(w.grid, acc_o, w.threshold)
        lo, hi_ = np.searchsorted(ev, e), np.searchsorted(ev, e, side="right")
        pk = res.peaks[lo:hi_].cpu().numpy().view(np.int32).reshape(-1, 5).copy().view(oracle_mod.PEAK_DTYPE).reshape(-1)
        pk_o["event"] = e
        assert np.array_equal(pk, pk_o), e
        if len(pk_o):
            rng = np.random.default_rng(e)
            sel = np.sort(rng.choice(len(pk_o), min(150, len(pk_o)), replace=False))
            po_o, hi_o = oracle_mod.associate(w.grid, b.x, b.y, b.event_offsets, pk_o[sel], w.window)
            for t, p in enumerate(sel):
                a0, a1 = int(po_all[lo + p]), int(po_all[lo + p + 1])
                got = res.hit_idx[a0:a1].cpu().numpy()
                assert np.array_equal(got, hi_o[po_o[t]:po_o[t + 1]]), (e, p)
    # accumulators of the sampled events from a plain vote of the whole batch
    ctx.vote(hits)
    for e in sample[:3]:
        be = b.event(e)
        assert np.array_equal(ctx.accumulator(e), oracle_mod.vote(w.grid, be.x, be.y)[0]), e
    ctx.close()


def test_pileup_events_sampled_columns(ht, oracle_mod):
    """80k-hit events on the 1024 x 128 x 512 grid, in waves of one event."""
    w = synth.WORKLOADS["pileup_64x5000trk"]
    b = synth.generate(w, n_events=2)
    g = w.grid
    ctx = ht.Context(g, w.spec.layers)
    ctx.vote(ht.Hits.from_batch(b.event(1), device="cuda"))
    acc = ctx.accumulator(0)
    ctx.close()
    be = b.event(1)
    rng = np.random.default_rng(2)
    for _ in range(48):
        i, j = int(rng.integers(0, g.n_phi)), int(rng.integers(0, g.n_d0))
        assert np.array_equal(acc[i, j], oracle_mod.vote_column(g, be.x, be.y, i, j)), (i, j)
    pk_o1 = oracle_mod.peaks(g, acc[None], w.threshold)
    cells = g.n_phi * g.n_d0 * g.n_kappa
    pk, po, hi = _run(ht, g, b, w.threshold, w.window, budget=cells * 4, peak_cap=1 << 24, pair_cap=1 << 30)
    got1 = pk[pk["event"] == 1]
    pk_o1["event"] = 1
    assert np.array_equal(got1, pk_o1)
    base = int(np.searchsorted(pk["event"], 1))
    sel = np.sort(rng.choice(len(pk_o1), 60, replace=False))
    po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o1[sel], w.window)
    for t, p in enumerate(sel):
        assert np.array_equal(hi[po[base + p]:po[base + p + 1]], hi_o[po_o[t]:po_o[t + 1]])


@pytest.mark.parametrize("grid", [synth.Grid(96, 24, 64, -25.0, 25.0, -0.0114, 0.0114),
                                  synth.Grid(50, 17, 40, -7.0, 30.0, -0.02, 0.005),
                                  synth.Grid(40, 9, 32, -10.0, 10.0, 0.001, 0.02)])
def test_pruned_vote_equals_full_vote(ht, oracle_mod, grid):
    """Voting only each row's d0 band gives the full vote's accumulator
    (asymmetric ranges; a kappa range that does not straddle 0 disables pruning)."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=3, first_event=21)
    accs = []
    for prune in (3, 0):
        ctx = ht.Context(grid, w.spec.layers)
        ctx.set_option(ht.HT_OPT_PRUNE, prune)
        ctx.vote(ht.Hits.from_batch(b, device="cuda"))
        accs.append([ctx.accumulator(e) for e in range(3)])
        ctx.close()
    acc_o = oracle_mod.vote(grid, b.x, b.y, b.event_offsets)
    for e in range(3):
        assert np.array_equal(accs[0][e], accs[1][e])
        assert np.array_equal(accs[0][e], acc_o[e])
    # association over bands gives the same CSR
    outs = [_run(ht, grid, b, 4, 1, opts=((ht.HT_OPT_PRUNE, pr),)) for pr in (3, 0)]
    for a, c in zip(*outs):
        assert np.array_equal(a, c)
    pk_o = oracle_mod.peaks(grid, acc_o, 4)
    assert np.array_equal(outs[0][0], pk_o)
    _check_csr_rows(oracle_mod, grid, b, *outs[0], 1, 300)


@pytest.mark.parametrize("n_phi", [1, 2, 3])
def test_peaks_with_few_phi_rows(ht, oracle_mod, n_phi):
    """phi wraps onto the same rows: neighbours coincide (two rows) or are the
    cell itself (one row); the peak list must still follow the rule."""
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w, n_events=2)
    g = synth.Grid(n_phi, 6, 24, -10.0, 10.0, -0.0114, 0.0114)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    for thr in (1, 3):
        pk_o = oracle_mod.peaks(g, acc_o, thr)
        pk, po, hi = _run(ht, g, b, thr, 1)
        assert np.array_equal(pk, pk_o), (n_phi, thr)
        po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o, 1)
        assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o)


def test_association_windows(ht, oracle_mod):
    """Windows 0, 2, 3 and 6 at a low threshold: hits whose window holds two
    or more peaks of a column, ranked over one to four rounds of peaks."""
    w = synth.WORKLOADS["dense_event_500trk"]
    b = synth.generate(w, n_events=1)
    g = synth.Grid(48, 12, 64, -25.0, 25.0, -0.0114, 0.0114)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 3)
    for window in (0, 2, 3, 6):
        pk, po, hi = _run(ht, g, b, 3, window)
        assert np.array_equal(pk, pk_o)
        po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o, window)
        assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o), window


def test_association_passes(ht, oracle_mod):
    """Threshold 1 on a 512-bin kappa axis: a row's 32-column block holds more
    peaks than the 512 row cursors a warp keeps for this grid, so the block
    is walked in several passes."""
    w = synth.WORKLOADS["dense_event_500trk"]
    b = synth.generate(w, n_events=1)
    g = synth.Grid(16, 32, 512, -25.0, 25.0, -0.0114, 0.0114)
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 1)
    per_row = np.bincount(pk_o["i_phi"], minlength=g.n_phi)
    assert per_row.max() > 512
    pk, po, hi = _run(ht, g, b, 1, 1, pair_cap=1 << 28)
    assert np.array_equal(pk, pk_o)
    win = np.array([acc_o[0, p["i_phi"], p["i_d0"], max(p["i_kappa"] - 1, 0):p["i_kappa"] + 2].sum()
                    for p in pk_o], np.int64)
    assert np.array_equal(np.diff(po), win)
    _check_csr_rows(oracle_mod, g, b, pk, po, hi, 1, 1500)


def test_association_cursor_passes_point(ht, oracle_mod):
    """32 row cursors per warp against ~70 peaks per 32-column block: every
    block is walked in passes, with the same CSR as with the default."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=3, first_event=60)
    g = w.grid
    full = _run(ht, g, b, w.threshold, 1)
    small = _run(ht, g, b, w.threshold, 1, opts=((ht.HT_OPT_ASSOC_CURSORS, 32),))
    for a, c in zip(full, small):
        assert np.array_equal(a, c)
    _check_csr_rows(oracle_mod, g, b, *small, 1, 400)


def test_overflow_across_waves(ht):
    """Caps hit in the first wave: later waves lie wholly past the caps; the
    stored prefix and the true counts must match an unbounded run."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=6, first_event=300)
    g = synth.Grid(64, 16, 32, -25.0, 25.0, -0.0114, 0.0114)
    cells = g.n_phi * g.n_d0 * g.n_kappa
    full = _run(ht, g, b, 5, 1)
    for pc, qc in ((50, 400), (len(full[0]) // 3, len(full[2]) // 4)):
        ctx = ht.Context(g, w.spec.layers)
        ctx.set_option(ht.HT_OPT_ACC_BUDGET, 2 * cells * 4)
        res = ht.Results(pc, qc, device="cuda")
        ctx.process(ht.Hits.from_batch(b, device="cuda"), 5, 1, res)
        with pytest.raises(ht.HtError) as ei:
            ctx.sync()
        assert ei.value.status == ht.HT_ERR_OVERFLOW
        cnt = res.counts.cpu().numpy()
        assert cnt[0] == len(full[0]) and cnt[1] == len(full[2])
        pk, po, hi = res.host()
        assert np.array_equal(pk, full[0][:pc])
        n_ok = int(np.searchsorted(po, qc, side="right")) - 1   # rows ending at or below the cap
        assert np.array_equal(po[: n_ok + 1], full[1][: n_ok + 1])
        # every slot below the cap that belongs to a stored peak's row, the
        # crossing row's first hits included
        m = min(qc, int(full[1][len(pk)]))
        assert np.array_equal(hi[:m], full[2][:m])
        ctx.close()


@pytest.mark.parametrize("grid", [synth.WORKLOADS["batch_4096_lognormal"].grid,
                                  synth.Grid(96, 24, 64, -25.0, 25.0, -0.0114, 0.0114),
                                  synth.Grid(50, 17, 40, -7.0, 30.0, -0.02, 0.005)])
def test_vote_items_equal_hull_vote(ht, oracle_mod, grid):
    """The band vote over (hit, column) items gives the accumulators of the
    hull vote and of the oracle, and the same CSR with and without records."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=4, first_event=33)
    accs = []
    for items in (1, 0):
        ctx = ht.Context(grid, w.spec.layers)
        ctx.set_option(ht.HT_OPT_VOTE_ITEMS, items)
        assert ctx.get_option(ht.HT_OPT_VOTE_ITEMS) == items
        ctx.vote(ht.Hits.from_batch(b, device="cuda"))
        accs.append([ctx.accumulator(e) for e in range(b.n_events)])
        ctx.close()
    acc_o = oracle_mod.vote(grid, b.x, b.y, b.event_offsets)
    for e in range(b.n_events):
        assert np.array_equal(accs[0][e], acc_o[e]) and np.array_equal(accs[1][e], acc_o[e])
    outs = [_run(ht, grid, b, 5, 1, opts=((ht.HT_OPT_VOTE_ITEMS, it), (ht.HT_OPT_RECORDS, rec)))
            for it, rec in ((1, 1), (0, 1), (1, 0))]
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)
    assert np.array_equal(outs[0][0], oracle_mod.peaks(grid, acc_o, 5))
    _check_csr_rows(oracle_mod, grid, b, *outs[0], 1, 300)


def test_staged_hit_blocks_equal_direct_loads(ht, oracle_mod):
    """Hits copied into shared memory in 512-hit blocks (bulk copies) give the
    accumulators and CSR of direct loads: ragged events (block starts not
    16-byte aligned, one- to three-hit events with no bulk part, events of
    many blocks), with and without records, and a misaligned hit array
    (which falls back to direct loads)."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    parts = [synth.generate(w, n_events=5, first_event=70)]
    tiny = synth.generate(synth.WORKLOADS["single_event_10trk"], n_events=3)
    xs = [parts[0].x] + [tiny.x[:k] for k in (1, 3, 2)]
    ys = [parts[0].y] + [tiny.y[:k] for k in (1, 3, 2)]
    sizes = list(np.diff(parts[0].event_offsets)) + [1, 3, 2]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    b = synth.from_arrays(np.concatenate(xs), np.concatenate(ys), event_offsets=offs)
    g = w.grid
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    outs = []
    for staging, rec in ((1, 1), (0, 1), (1, 0)):
        opts = ((ht.HT_OPT_HIT_STAGING, staging), (ht.HT_OPT_RECORDS, rec), (ht.HT_OPT_TILE_PHI, 4),
                (ht.HT_OPT_TILE_D0, 16), (ht.HT_OPT_THREADS, 128))
        outs.append(_run(ht, g, b, w.threshold, w.window, opts=opts))
        ctx = ht.Context(g, w.spec.layers)
        for k, v in opts:
            ctx.set_option(k, v)
        assert ctx.get_option(ht.HT_OPT_HIT_STAGING) == staging
        ctx.vote(ht.Hits.from_batch(b, device="cuda"))
        for e in range(b.n_events):
            assert np.array_equal(ctx.accumulator(e), acc_o[e]), (staging, rec, e)
        ctx.close()
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)
    assert np.array_equal(outs[0][0], oracle_mod.peaks(g, acc_o, w.threshold))
    _check_csr_rows(oracle_mod, g, b, *outs[0], w.window, 300)
    # hit arrays 4 bytes off a 16-byte boundary: direct loads, same result
    xb = torch.zeros(b.n_hits + 1, dtype=torch.float32, device="cuda")
    yb = torch.zeros(b.n_hits + 1, dtype=torch.float32, device="cuda")
    xb[1:] = torch.from_numpy(b.x).cuda()
    yb[1:] = torch.from_numpy(b.y).cuda()
    hits = ht.Hits.from_batch(b, device="cuda")
    hits.arrays = (xb[1:], yb[1:]) + tuple(hits.arrays[2:])
    hits.struct.x, hits.struct.y = xb[1:].data_ptr(), yb[1:].data_ptr()
    ctx = ht.Context(g, w.spec.layers)
    ctx.set_option(ht.HT_OPT_HIT_STAGING, 1)
    res = ht.Results(1 << 22, 1 << 27, device="cuda")
    ctx.process(hits, w.threshold, w.window, res)
    ctx.sync()
    for a, c in zip(outs[0], res.host()):
        assert np.array_equal(a, c)
    ctx.close()


def test_band_split_equals_oracle(ht, oracle_mod):
    """Narrow-band hits queued apart and walking their own bands give the
    accumulators, records, peaks and rows of one hull queue and of the
    oracle: splits 0 (one queue), auto, 3, every band narrow (16, 256), with
    and without records, 4 x 16 and 8 x 8 tiles, a ragged 4 x 12 tile, and
    events of one to three hits (partial rings merged into one batch)."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    part = synth.generate(w, n_events=4, first_event=90)
    tiny = synth.generate(synth.WORKLOADS["single_event_10trk"], n_events=3)
    xs = [part.x] + [tiny.x[:k] for k in (1, 3, 2)]
    ys = [part.y] + [tiny.y[:k] for k in (1, 3, 2)]
    sizes = list(np.diff(part.event_offsets)) + [1, 3, 2]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    b = synth.from_arrays(np.concatenate(xs), np.concatenate(ys), event_offsets=offs)
    g = w.grid
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    ref = None
    for tp, td in ((4, 16), (8, 8), (4, 12)):
        for split in (0, -1, 3, 16, 256):
            for rec in (1, 0):
                if rec == 0 and split not in (0, -1):
                    continue
                opts = ((ht.HT_OPT_BAND_SPLIT, split), (ht.HT_OPT_RECORDS, rec), (ht.HT_OPT_TILE_PHI, tp),
                        (ht.HT_OPT_TILE_D0, td), (ht.HT_OPT_THREADS, 128))
                out = _run(ht, g, b, w.threshold, w.window, opts=opts)
                if ref is None:
                    ref = out
                else:
                    for a, c in zip(ref, out):
                        assert np.array_equal(a, c), (tp, td, split, rec)
                ctx = ht.Context(g, w.spec.layers)
                for k, v in opts:
                    ctx.set_option(k, v)
                want = {0: 0, -1: max(3, td * 5 // 16)}.get(split, split)
                assert ctx.get_option(ht.HT_OPT_BAND_SPLIT) == want
                ctx.vote(ht.Hits.from_batch(b, device="cuda"))
                for e in range(b.n_events):
                    assert np.array_equal(ctx.accumulator(e), acc_o[e]), (tp, td, split, rec, e)
                ctx.close()
    assert np.array_equal(ref[0], oracle_mod.peaks(g, acc_o, w.threshold))
    _check_csr_rows(oracle_mod, g, b, *ref, w.window, 300)
    # the option's range
    ctx = ht.Context(g, w.spec.layers)
    with pytest.raises(ht.HtError):
        ctx.set_option(ht.HT_OPT_BAND_SPLIT, -2)
    ctx.close()
