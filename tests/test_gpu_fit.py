"""GPU parity of the circle fit (ht_fit) against the oracle: every field of
every stored candidate's fit must be equal bit for bit."""

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


FIELDS = ("status", "n_hits", "cos_phi0", "sin_phi0", "d0", "kappa", "chi2")


def _same(a, b):
    assert a.shape == b.shape
    for f in FIELDS:
        assert np.array_equal(a[f], b[f]), f


@pytest.mark.parametrize("mode", ["point", "range"])
def test_fit_equals_oracle_device_and_host(ht, oracle_mod, mode):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    g = w.grid if mode == "point" else synth.Grid(64, 16, 64, -25.0, 25.0, -0.0114, 0.0114)
    b = synth.generate(w, n_events=3, first_event=5)
    ctx = ht.Context(g, w.spec.layers)
    if mode == "range":
        ctx.set_option(ht.HT_OPT_VOTE_MODE, ht.HT_VOTE_RANGE)
    thr = w.threshold if mode == "point" else 14
    # device results
    res = ht.Results(1 << 20, 1 << 26, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), thr, 1, res)
    ctx.sync()
    pk, po, hi = res.host()
    fits_d = ctx.fit(res)
    torch.cuda.synchronize()
    fd = ht.tracks_host(fits_d, len(pk))
    want = oracle_mod.fit(g, b.x, b.y, pk, po, hi)
    assert (want["status"] == 1).sum() > 100
    _same(fd.view(oracle_mod.TRACK_DTYPE), want)
    # host results from host hits
    rh = ht.Results(1 << 20, 1 << 26)
    ctx.process(ht.Hits.from_batch(b), thr, 1, rh)
    fh = ctx.fit(rh)
    _same(fh.view(oracle_mod.TRACK_DTYPE), want)
    ctx.close()


def test_fit_marks_rows_cut_by_the_pair_cap(ht, oracle_mod):
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w, n_events=3, first_event=8)
    g = w.grid
    ctx = ht.Context(g, w.spec.layers)
    ctx.set_option(ht.HT_OPT_VOTE_MODE, ht.HT_VOTE_RANGE)
    full = ht.Results(1 << 16, 1 << 22, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), 8, 1, full)
    ctx.sync()
    pk, po, hi = full.host()
    qc = int(po[len(pk) // 2]) + 3  # cuts the row that holds pair qc - 1
    cut = ht.Results(1 << 16, qc, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), 8, 1, cut)
    with pytest.raises(ht.HtError):
        ctx.sync()
    f = ht.tracks_host(ctx.fit(cut), len(pk))
    want = oracle_mod.fit(g, b.x, b.y, pk, po, hi)
    whole = po[1:] <= qc
    _same(f[whole].view(oracle_mod.TRACK_DTYPE), want[whole])
    assert np.all(f["status"][~whole] == -1)
    assert np.array_equal(f["n_hits"][~whole], (po[1:] - po[:-1])[~whole])
    ctx.close()


def test_fit_needs_a_processed_batch(ht):
    g = synth.WORKLOADS["single_event_10trk"].grid
    ctx = ht.Context(g, synth.LAYERS_13)
    res = ht.Results(16, 16)
    with pytest.raises(ht.HtError) as ei:
        ctx.fit(res)
    assert ei.value.status == ht.HT_ERR_STATE
    ctx.close()
