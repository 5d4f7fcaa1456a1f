"""The GPU's float32 and double-float stages never decide a bin the binary64
definition disagrees with.

Uses the numpy model in filter_model.py (a restatement of the kernels'
arithmetic) with the reciprocal error pushed to both ends of its bound, on
cells sampled from every workload grid plus adversarial cells: hits next to
a perigee point (tiny denominators) and hits on circles whose curvature is
exactly a bin edge.
"""

import math

import numpy as np
import pytest

import filter_model as fm
from paper_1311_2769_gb300 import synth


def _cells(oracle_mod, wname, n, seed):
    w = synth.WORKLOADS[wname]
    g = w.grid
    b = synth.generate(w, n_events=1, first_event=seed)
    c, s, d = oracle_mod.tables(g)
    rng = np.random.default_rng(seed)
    h = rng.integers(0, b.n_hits, n)
    i = rng.integers(0, g.n_phi, n)
    j = rng.integers(0, g.n_d0, n)
    return g, b.x[h], b.y[h], c[i], s[i], d[j]


def _near_perigee(oracle_mod, g, n, seed):
    c, s, d = oracle_mod.tables(g)
    rng = np.random.default_rng(seed)
    i = rng.integers(0, g.n_phi, n)
    j = rng.integers(0, g.n_d0, n)
    px = -d[j].astype(np.float64) * s[i]
    py = d[j].astype(np.float64) * c[i]
    dist = 10.0 ** rng.uniform(-6, 1, n)
    ang = rng.uniform(0, 2 * math.pi, n)
    x = (px + dist * np.cos(ang)).astype(np.float32)
    y = (py + dist * np.sin(ang)).astype(np.float32)
    return x, y, c[i], s[i], d[j]


def _on_bin_edges(oracle_mod, g, n, seed):
    c, s, d = oracle_mod.tables(g)
    rng = np.random.default_rng(seed)
    i = rng.integers(0, g.n_phi, n)
    j = rng.integers(0, g.n_d0, n)
    k = rng.integers(0, g.n_kappa + 1, n)
    kmin, kmax = float(np.float32(g.kappa_min)), float(np.float32(g.kappa_max))
    kap = kmin + k * (kmax - kmin) / g.n_kappa
    kap = np.where(kap == 0, 1e-9, kap)
    phi0 = np.arctan2(s[i].astype(np.float64), c[i].astype(np.float64))
    x, y, _, ok = synth.helix_hits(phi0, d[j].astype(np.float64), kap, synth.LAYERS_13)
    lay = rng.integers(0, len(synth.LAYERS_13), n)
    sel = ok[np.arange(n), lay]
    return (x[np.arange(n), lay][sel].astype(np.float32), y[np.arange(n), lay][sel].astype(np.float32),
            c[i][sel], s[i][sel], d[j][sel])


@pytest.mark.parametrize("wname", ["single_event_10trk", "dense_event_500trk", "batch_4096_lognormal",
                                   "pileup_64x5000trk"])
def test_stage1_and_stage2_never_disagree_with_binary64(oracle_mod, wname):
    g, x, y, c, s, d = _cells(oracle_mod, wname, 400_000, 7)
    parts = [(x, y, c, s, d), _near_perigee(oracle_mod, g, 100_000, 8), _on_bin_edges(oracle_mod, g, 100_000, 9)]
    x, y, c, s, d = (np.concatenate([p[t] for p in parts]) for t in range(5))
    K = fm.consts(g, oracle_mod.tables(g)[2])
    ref = oracle_mod.kbin_cells(g, x, y, c, s, d).astype(np.int64)
    n0 = 400_000
    und1 = und2 = und2_adv = 0
    for err in (-fm.ER, 0.0, fm.ER):
        k1 = fm.stage1(x, y, c, s, d, K, err)
        dec = k1 != -2
        bad = np.nonzero(dec & (k1 != ref))[0]
        assert bad.size == 0, f"stage 1 wrong on {bad.size} cells, e.g. {[(x[t], y[t], c[t], s[t], d[t], k1[t], ref[t]) for t in bad[:3]]}"
        k2 = fm.stage2(x, y, c, s, d, K, err)
        dec2 = k2 != -2
        bad2 = np.nonzero(dec2 & (k2 != ref))[0]
        assert bad2.size == 0, f"stage 2 wrong on {bad2.size} cells, e.g. {[(x[t], y[t], c[t], s[t], d[t], k2[t], ref[t]) for t in bad2[:3]]}"
        und1 = max(und1, int((~dec[:n0]).sum()))
        und2 = max(und2, int((~dec2[:n0] & ~dec[:n0]).sum()))
        und2_adv = max(und2_adv, int((~dec2[n0:] & ~dec[n0:]).sum()))
    # on ordinary cells the float32 stage decides almost everything
    assert und1 / n0 < 2e-3, und1
    # and the double-float stage leaves essentially nothing to binary64
    assert und2 <= 2, und2
    # even among adversarial cells only hits within ~1e-3 cm of a perigee point reach binary64
    assert und2_adv / (x.shape[0] - n0) < 0.7, und2_adv


@pytest.mark.parametrize("wname", ["single_event_10trk", "dense_event_500trk", "batch_4096_lognormal",
                                   "pileup_64x5000trk"])
def test_d0_band_contains_every_voting_column(oracle_mod, wname):
    """The pruned vote evaluates only the d0 band of each (hit, phi row); every
    column where the hit votes in binary64 must lie inside it, also with the
    band's roots pushed beyond the errors of the approximate square roots and
    reciprocals the kernels use."""
    w = synth.WORKLOADS[wname]
    g = w.grid
    b = synth.generate(w, n_events=1, first_event=5)
    c, s, d = oracle_mod.tables(g)
    C = fm.band_consts(g, d)
    rng = np.random.default_rng(1)
    nh = min(600, b.n_hits)
    hs = rng.choice(b.n_hits, nh, replace=False)
    rows = rng.choice(g.n_phi, min(64, g.n_phi), replace=False)
    x = np.repeat(b.x[hs], len(rows))
    y = np.repeat(b.y[hs], len(rows))
    ci = np.tile(c[rows], nh)
    si = np.tile(s[rows], nh)
    frac = []
    tilts = ((0, 0, 0, 0), (1, 1, 1, 1), (-1, -1, -1, -1), (1, -1, -1, 1), (-1, 1, 1, -1))
    for j0, nj in ((0, g.n_d0), (0, max(1, g.n_d0 // 2)), (g.n_d0 // 4, max(1, g.n_d0 // 4))):
        votes = {j: oracle_mod.kbin_cells(g, x, y, ci, si, np.full(x.shape, d[j], np.float32)) >= 0
                 for j in range(j0, j0 + nj)}
        for tilt in tilts:
            jlo, jhi = fm.band(x, y, ci, si, j0, nj, d, C, tilt)
            for j in range(j0, j0 + nj):
                outside = votes[j] & ((j < jlo) | (j > jhi))
                assert not outside.any(), (tilt, j, np.nonzero(outside)[0][:5])
            if tilt == tilts[0]:
                frac.append(np.maximum(jhi - jlo + 1, 0).mean() / nj)
    assert frac[0] < 0.45, frac
