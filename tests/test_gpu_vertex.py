"""GPU parity of the second Hough transform (ht_vertices) against the oracle:
the vertex list of the candidates of an ht_process must equal the oracle's."""

import collections
import math

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VG = collections.namedtuple("VG", "n_x n_y x_min x_max y_min y_max")
LINE_GRID = synth.Grid(256, 64, 1, -40.0, 40.0, -0.0005, 0.0005)


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_2769_gb300 import build, ht as mod
    build.build()
    mod.load()
    return mod


def _jets(rng, n_events):
    """Events of four displaced jets of straight tracks (the paper's picture)."""
    xs, ys, offs, verts = [], [], [0], []
    for _ in range(n_events):
        vs = rng.uniform(-20, 20, (4, 2))
        phi0, d0, kap = [], [], []
        for xv, yv in vs:
            axis = math.atan2(yv, xv)
            for _ in range(8):
                psi = axis + rng.uniform(-0.6, 0.6)
                phi0.append(psi % (2 * math.pi))
                d0.append(yv * math.cos(psi) - xv * math.sin(psi))
                kap.append(rng.uniform(-1e-5, 1e-5))
        x, y, _, ok = synth.helix_hits(phi0, d0, kap, synth.LAYERS_13)
        xs.append(x[ok].astype(np.float32))
        ys.append(y[ok].astype(np.float32))
        offs.append(offs[-1] + xs[-1].shape[0])
        verts.append(vs)
    return synth.from_arrays(np.concatenate(xs), np.concatenate(ys), event_offsets=np.array(offs, np.int32)), verts


def _process(ht, g, b, thr, device=True):
    ctx = ht.Context(g, synth.LAYERS_13)
    res = ht.Results(1 << 18, 1 << 24, device="cuda" if device else None)
    ctx.process(ht.Hits.from_batch(b, device="cuda" if device else None), thr, 1, res)
    if device:
        ctx.sync()
    return ctx, res


def test_displaced_jets_vertices_equal_oracle(ht, oracle_mod):
    rng = np.random.default_rng(3)
    b, verts = _jets(rng, 4)
    vg = VG(64, 64, -32.0, 32.0, -32.0, 32.0)
    ctx, res = _process(ht, LINE_GRID, b, 9)
    pk, _, _ = res.host()
    want = oracle_mod.vertex_peaks(vg, oracle_mod.vertex_vote(LINE_GRID, vg, pk, b.n_events), 6)
    out, cnt = ctx.vertices(vg, res, 6)
    got = ht.vertices_host(out, int(cnt.item()))
    assert np.array_equal(got.view(oracle_mod.VERTEX_DTYPE), want)
    # every true vertex has a found vertex within two cells
    for e, vs in enumerate(verts):
        ev = got[got["event"] == e]
        for xv, yv in vs:
            a, c = int((xv + 32.0) // 1.0), int((yv + 32.0) // 1.0)
            assert np.any((np.abs(ev["i_x"] - a) <= 2) & (np.abs(ev["i_y"] - c) <= 2)), (e, xv, yv)
    ctx.close()
    # the same through host results
    ctx, rh = _process(ht, LINE_GRID, b, 9, device=False)
    gh, n = ctx.vertices(vg, rh, 6)
    assert n == len(want) and np.array_equal(gh.view(oracle_mod.VERTEX_DTYPE), want)
    ctx.close()


def test_vertices_on_batch_candidates_equal_oracle(ht, oracle_mod):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=2, first_event=9)
    vg = VG(96, 80, -37.0, 29.0, -20.5, 44.0)
    ctx, res = _process(ht, w.grid, b, w.threshold)
    pk, _, _ = res.host()
    want = oracle_mod.vertex_peaks(vg, oracle_mod.vertex_vote(w.grid, vg, pk, b.n_events), 40)
    assert len(want) > 10
    out, cnt = ctx.vertices(vg, res, 40)
    assert int(cnt.item()) == len(want)
    got = ht.vertices_host(out, len(want))
    assert np.array_equal(got.view(oracle_mod.VERTEX_DTYPE), want)
    # a small cap keeps the prefix and the true count
    small, cnt2 = ctx.vertices(vg, res, 40, cap=5)
    torch.cuda.synchronize()
    assert int(cnt2.item()) == len(want)
    assert np.array_equal(ht.vertices_host(small, 5).view(oracle_mod.VERTEX_DTYPE), want[:5])
    ctx.close()
