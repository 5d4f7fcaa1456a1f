"""GPU parity of line voting (HT_VOTE_LINE, the paper's kappa = 0 model)
against the oracle: accumulators, peaks and association CSR bit for bit."""

import math

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRIDS = [synth.Grid(256, 64, 1, -40.0, 40.0, -0.0005, 0.0005),
         synth.Grid(37, 45, 1, -31.0, 23.0, -0.001, 0.002)]


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_2769_gb300 import build, ht as mod
    build.build()
    mod.load()
    return mod


def _events(rng, n_events, n_tracks=15, noise=40):
    xs, ys, offs = [], [], [0]
    for _ in range(n_events):
        phi0 = rng.uniform(0, 2 * math.pi, n_tracks)
        d0 = rng.uniform(-20, 20, n_tracks)
        x, y, _, ok = synth.helix_hits(phi0, d0, np.full(n_tracks, 1e-9), synth.LAYERS_13)
        r = np.asarray(synth.LAYERS_13)[rng.integers(0, 13, noise)]
        a = rng.uniform(0, 2 * math.pi, noise)
        xs.append(np.concatenate([x[ok], r * np.cos(a)]).astype(np.float32))
        ys.append(np.concatenate([y[ok], r * np.sin(a)]).astype(np.float32))
        offs.append(offs[-1] + xs[-1].shape[0])
    return synth.from_arrays(np.concatenate(xs), np.concatenate(ys), event_offsets=np.array(offs, np.int32))


def _ctx(ht, g):
    ctx = ht.Context(g, synth.LAYERS_13)
    ctx.set_option(ht.HT_OPT_VOTE_MODE, ht.HT_VOTE_LINE)
    return ctx


@pytest.mark.parametrize("gi", [0, 1])
def test_line_vote_and_process_equal_oracle(ht, oracle_mod, gi):
    g = GRIDS[gi]
    b = _events(np.random.default_rng(gi), 3)
    acc_o = oracle_mod.vote_line(g, b.x, b.y, b.event_offsets)
    ctx = _ctx(ht, g)
    ctx.vote(ht.Hits.from_batch(b, device="cuda"))
    for e in range(b.n_events):
        assert np.array_equal(ctx.accumulator(e), acc_o[e]), e
    pk_o = oracle_mod.peaks(g, acc_o, 7)
    assert len(pk_o) >= 10
    for window in (0, 1, 2):
        res = ht.Results(1 << 16, 1 << 22, device="cuda")
        ctx.process(ht.Hits.from_batch(b, device="cuda"), 7, window, res)
        ctx.sync()
        pk, po, hi = res.host()
        po_o, hi_o = oracle_mod.associate_line(g, b.x, b.y, b.event_offsets, pk_o, window)
        assert np.array_equal(pk, pk_o)
        assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o), window
    ctx.close()


def test_line_host_calls_and_grid_check(ht, oracle_mod):
    g = GRIDS[0]
    b = _events(np.random.default_rng(5), 2)
    ctx = _ctx(ht, g)
    ctx.vote(ht.Hits.from_batch(b))
    pk = ctx.peaks(7)
    acc_o = oracle_mod.vote_line(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 7)
    assert np.array_equal(pk, pk_o)
    po, hi = ctx.associate(1, len(pk))
    po_o, hi_o = oracle_mod.associate_line(g, b.x, b.y, b.event_offsets, pk_o, 1)
    assert np.array_equal(po, po_o) and np.array_equal(hi, hi_o)
    ctx.close()
    ctx = ht.Context(synth.WORKLOADS["single_event_10trk"].grid, synth.LAYERS_13)
    with pytest.raises(ht.HtError) as ei:
        ctx.set_option(ht.HT_OPT_VOTE_MODE, ht.HT_VOTE_LINE)
    assert ei.value.status == ht.HT_ERR_INVALID_ARG
    ctx.close()


def test_curved_through_origin_grid_equals_oracle(ht, oracle_mod):
    """The paper's other two-parameter model, curved tracks from the origin
    (d0 = 0), is the point vote on a grid with one d0 bin centred on 0."""
    g = synth.Grid(128, 1, 64, -1.0, 1.0, -0.0114, 0.0114)
    rng = np.random.default_rng(8)
    xs, ys, offs = [], [], [0]
    for _ in range(3):
        n = 12
        x, y, _, ok = synth.helix_hits(rng.uniform(0, 2 * math.pi, n), np.zeros(n),
                                       rng.uniform(0.002, 0.009, n) * rng.choice([-1.0, 1.0], n), synth.LAYERS_13)
        xs.append(x[ok].astype(np.float32))
        ys.append(y[ok].astype(np.float32))
        offs.append(offs[-1] + xs[-1].shape[0])
    b = synth.from_arrays(np.concatenate(xs), np.concatenate(ys), event_offsets=np.array(offs, np.int32))
    acc_o = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk_o = oracle_mod.peaks(g, acc_o, 8)
    assert len(pk_o) >= 10
    po_o, hi_o = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk_o, 1)
    ctx = ht.Context(g, synth.LAYERS_13)
    res = ht.Results(1 << 14, 1 << 20, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), 8, 1, res)
    ctx.sync()
    pk, po, hi = res.host()
    assert np.array_equal(pk, pk_o) and np.array_equal(po, po_o) and np.array_equal(hi, hi_o)
    ctx.close()
