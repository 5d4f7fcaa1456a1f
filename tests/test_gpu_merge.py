"""GPU parity of duplicate and mirror merging (ht_merge) against the oracle:
every candidate's state and the kept count must be equal."""

import collections

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


def _run(ht, oracle_mod, g, b, thr, window, radii, mode=None, device=True):
    ctx = ht.Context(g, b.layer_r)
    if mode is not None:
        ctx.set_option(ht.HT_OPT_VOTE_MODE, mode)
    dev = "cuda" if device else None
    res = ht.Results(1 << 20, 1 << 26, device=dev)
    ctx.process(ht.Hits.from_batch(b, device=dev), thr, window, res)
    if device:
        ctx.sync()
    pk, po, hi = res.host()
    fits = ctx.fit(res)
    fits_h = ht.tracks_host(fits, len(pk)) if device else fits
    want_fits = oracle_mod.fit(g, b.x, b.y, pk, po, hi)
    assert np.array_equal(fits_h.view(oracle_mod.TRACK_DTYPE)["status"], want_fits["status"])
    for r in radii:
        want, kept_o = oracle_mod.merge(g, b.x, b.y, pk, po, hi, want_fits, r)
        state, kept = ctx.merge(res, fits, r)
        if device:
            torch.cuda.synchronize()
            state, kept = state[: len(pk)].cpu().numpy(), int(kept.item())
        assert np.array_equal(state, want), r
        assert kept == kept_o, r
    ctx.close()
    return pk


@pytest.mark.parametrize("device", [True, False])
def test_merge_equals_oracle_batch_events(ht, oracle_mod, device):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=3, first_event=11)
    pk = _run(ht, oracle_mod, w.grid, b, w.threshold, 1, (2, 0, 3), device=device)
    assert len(pk) > 10000


def test_merge_wraps_phi_on_a_small_grid(ht, oracle_mod):
    """n_phi = 4: at radius 2 every phi0 row is within reach (each once)."""
    g = synth.Grid(4, 16, 64, -20.0, 20.0, -0.0114, 0.0114)
    b = synth.generate(synth.WORKLOADS["batch_4096_lognormal"], n_events=2, first_event=2)
    _run(ht, oracle_mod, g, b, 20, 1, (1, 2, 5))


def test_merge_of_line_voted_candidates(ht, oracle_mod):
    """Straight displaced tracks voted as lines (one kappa bin)."""
    g = synth.Grid(256, 64, 1, -40.0, 40.0, -0.0005, 0.0005)
    rng = np.random.default_rng(4)
    xs, ys, offs = [], [], [0]
    for _ in range(3):
        phi0 = rng.uniform(0, 2 * np.pi, 20)
        d0 = rng.uniform(-20, 20, 20)
        x, y, _, ok = synth.helix_hits(phi0, d0, np.full(20, 1e-9), synth.LAYERS_13)
        xs.append(x[ok].astype(np.float32))
        ys.append(y[ok].astype(np.float32))
        offs.append(offs[-1] + xs[-1].shape[0])
    b = synth.from_arrays(np.concatenate(xs), np.concatenate(ys), event_offsets=np.array(offs, np.int32))
    _run(ht, oracle_mod, g, b, 7, 1, (2, 4), mode=ht.HT_VOTE_LINE)


def test_merge_marks_rows_cut_by_the_pair_cap_unfitted(ht, oracle_mod):
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w, n_events=3, first_event=8)
    g = w.grid
    ctx = ht.Context(g, w.spec.layers)
    full = ht.Results(1 << 16, 1 << 22, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), 4, 1, full)
    ctx.sync()
    pk, po, hi = full.host()
    qc = int(po[len(pk) // 2]) + 3
    cut = ht.Results(1 << 16, qc, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), 4, 1, cut)
    with pytest.raises(ht.HtError):
        ctx.sync()
    fits = ctx.fit(cut)
    state, kept = ctx.merge(cut, fits, 2)
    torch.cuda.synchronize()
    state = state[: len(pk)].cpu().numpy()
    f = ht.tracks_host(fits, len(pk)).view(oracle_mod.TRACK_DTYPE)
    want, kept_o = oracle_mod.merge(g, b.x, b.y, pk, po, hi, f, 2)
    assert np.all(state[po[1:] > qc] == ht.HT_MERGE_UNFITTED)
    assert np.array_equal(state, want) and int(kept.item()) == kept_o
    ctx.close()


def test_merge_argument_checks(ht):
    g = synth.WORKLOADS["single_event_10trk"].grid
    ctx = ht.Context(g, synth.LAYERS_13)
    res = ht.Results(1 << 12, 1 << 16)
    fits = np.zeros(16, ht.TRACK_DTYPE)
    with pytest.raises(ht.HtError) as ei:
        ctx.merge(res, fits, 2)
    assert ei.value.status == ht.HT_ERR_STATE
    b = synth.generate(synth.WORKLOADS["single_event_10trk"], n_events=1)
    ctx.process(ht.Hits.from_batch(b), 8, 1, res)
    for bad in (-1, 65):
        with pytest.raises(ht.HtError) as ei:
            ctx.merge(res, fits, bad)
        assert ei.value.status == ht.HT_ERR_INVALID_ARG
    ctx.close()
