"""Pins of the oracle's range voting (CPU only).

Range voting: in cell (i, j) a hit votes for every kappa bin from the lowest
to the highest bin of its curve at the cell's four corners (phi0 edges
m 2pi/n_phi, periodic; d0 edges d0_min + n (d0_max - d0_min)/n_d0), clipped
to the kappa range; a corner whose denominator is not positive leaves the
cell without a vote.  The pins below hold the oracle to properties fixed by
the geometry, not to a retyping of its own code.
"""

import math

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

C0 = synth.Grid(64, 8, 64, -10.0, 10.0, -0.0114, 0.0114)


def _cell_of(g, phi0, d0, kappa):
    i = int(math.floor((phi0 % (2 * math.pi)) / (2 * math.pi / g.n_phi)))
    j = int(math.floor((d0 - g.d0_min) / ((g.d0_max - g.d0_min) / g.n_d0)))
    k = int(math.floor((kappa - g.kappa_min) / ((g.kappa_max - g.kappa_min) / g.n_kappa)))
    return i, j, k


def _tracks(rng, n, g):
    phi0 = rng.uniform(0.0, 2 * math.pi, n)
    d0 = rng.uniform(0.8 * g.d0_min, 0.8 * g.d0_max, n)
    kap = rng.uniform(0.002, 0.009, n) * rng.choice([-1.0, 1.0], n)
    return phi0, d0, kap


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_off_centre_tracks_fill_their_cell(oracle_mod, seed):
    """Every hit of an unsmeared track lies on the curve through the track's
    own (phi0, d0, kappa), so under range voting the cell containing those
    parameters collects one vote per hit at the track's kappa bin (up to a
    neighbouring bin at a bin edge).  Point voting, which samples only the
    cell centre, generally does not."""
    g = C0
    rng = np.random.default_rng(seed)
    phi0, d0, kap = _tracks(rng, 10, g)
    x, y, _, ok = synth.helix_hits(phi0, d0, kap, synth.LAYERS_10)
    full_range = full_point = 0
    for t in range(10):
        hx, hy = x[t][ok[t]].astype(np.float32), y[t][ok[t]].astype(np.float32)
        n = hx.shape[0]
        i, j, k = _cell_of(g, phi0[t], d0[t], kap[t])
        ar = oracle_mod.vote_range(g, hx, hy)[0]
        ap = oracle_mod.vote(g, hx, hy)[0]
        ks = slice(max(k - 1, 0), min(k + 2, g.n_kappa))
        full_range += int(ar[i, j, ks].max() == n)
        full_point += int(ap[i, j, ks].max() == n)
    assert full_range >= 9, full_range
    assert full_point < full_range, (full_point, full_range)


def test_range_is_the_hull_of_corner_bins_by_sampling(oracle_mod):
    """Brute force on a small grid: bin every point of a 9 x 9 lattice over
    each cell (corners included) by the binary64 definition.  The range must
    equal the hull of the four corner bins, so it lies inside the lattice's
    hull, and equals it wherever the lattice's extremes sit on corners.  This
    catches a wrong corner, a missing phi wrap or a swapped edge."""
    g = synth.Grid(12, 4, 32, -6.0, 6.0, -0.0114, 0.0114)
    rng = np.random.default_rng(5)
    phi0, d0, kap = _tracks(rng, 3, g)
    x, y, _, ok = synth.helix_hits(phi0, d0, kap, synth.LAYERS_10)
    hx = np.concatenate([x[t][ok[t]] for t in range(3)]).astype(np.float32)[::3]
    hy = np.concatenate([y[t][ok[t]] for t in range(3)]).astype(np.float32)[::3]
    dphi = 2 * math.pi / g.n_phi
    dw = (g.d0_max - g.d0_min) / g.n_d0
    u = np.linspace(0.0, 1.0, 9)
    checked = equal = 0
    for h in range(hx.shape[0]):
        for i in range(g.n_phi):
            for j in range(g.n_d0):
                phis = (i + u) * dphi
                ds = np.array([np.float32(g.d0_min + (j + v) * dw) for v in u], np.float32)
                P, D = np.meshgrid(phis, ds, indexing="ij")
                c = np.cos(P).astype(np.float32)
                s = np.sin(P).astype(np.float32)
                codes = oracle_mod.code_cells(g, np.full(P.size, hx[h]), np.full(P.size, hy[h]),
                                              c.ravel(), s.ravel(), D.ravel()).reshape(P.shape)
                r = oracle_mod.range_of(g, hx[h], hy[h], i, j)
                if (codes == oracle_mod.UNDEF).any():
                    continue
                corners = codes[[0, -1, 0, -1], [0, 0, -1, -1]]
                lo, hi = int(corners.min()), int(corners.max())
                if hi < 0 or lo >= g.n_kappa:
                    assert r is None
                    continue
                assert r == (max(lo, 0), min(hi, g.n_kappa - 1)), (h, i, j)
                checked += 1
                assert codes.min() <= lo and codes.max() >= hi
                if codes.min() == lo and codes.max() == hi:
                    equal += 1
    assert checked > 50 and equal > 0.9 * checked, (checked, equal)


def test_range_contains_the_point_bin(oracle_mod):
    """The cell centre lies inside the cell, so where the curve's kappa is
    monotone over the cell (nearly everywhere) its centre bin lies between
    the corner bins: the range vote contains the point vote."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    g = w.grid
    b = synth.generate(w, n_events=1, first_event=7)
    rng = np.random.default_rng(3)
    hs = rng.choice(b.n_hits, 300, replace=False)
    cells = rng.integers(0, [g.n_phi, g.n_d0], size=(300, 2))
    n = inside = 0
    for h in hs:
        for i, j in cells:
            k = oracle_mod.kbin(g, b.x[h], b.y[h], i, j)
            if k < 0:
                continue
            r = oracle_mod.range_of(g, b.x[h], b.y[h], i, j)
            n += 1
            inside += int(r is not None and r[0] <= k <= r[1])
    assert n > 1000 and inside >= 0.999 * n, (n, inside)


def test_perigee_corner_leaves_its_cells_without_a_vote(oracle_mod):
    """A hit exactly at the perigee point of a corner (phi0 edge 0, d0 edge
    n) makes that corner's denominator zero: the four cells sharing the
    corner get no vote, while the hit still votes elsewhere."""
    g = C0
    _, _, de = oracle_mod.edges(g)
    n = 5
    hx, hy = np.float32(0.0), de[n]
    for i in (0, g.n_phi - 1):
        for j in (n - 1, n):
            assert oracle_mod.range_of(g, hx, hy, i, j) is None, (i, j)
    acc = oracle_mod.vote_range(g, np.array([hx]), np.array([hy]))[0]
    assert acc[0, n - 1].sum() == 0 and acc[g.n_phi - 1, n].sum() == 0
    assert acc.sum() > 0


def test_range_association_rows(oracle_mod):
    """Hit h joins peak (i, j, k) when its range in column (i, j) reaches
    within `window` of k; rows list hits in ascending order, and with window
    0 a row holds exactly the hits whose range contains k, as many as the
    peak's votes."""
    w = synth.WORKLOADS["single_event_10trk"]
    g = w.grid
    b = synth.generate(w)
    acc = oracle_mod.vote_range(g, b.x, b.y)
    pk = oracle_mod.peaks(g, acc, w.threshold)
    assert len(pk) > 0
    for window in (0, 1, 3):
        po, hi = oracle_mod.associate_range(g, b.x, b.y, b.event_offsets, pk, window)
        for p in range(min(len(pk), 60)):
            row = hi[po[p]:po[p + 1]]
            assert np.all(np.diff(row) > 0)
            want = []
            for h in range(b.n_hits):
                r = oracle_mod.range_of(g, b.x[h], b.y[h], pk["i_phi"][p], pk["i_d0"][p])
                if r is not None and r[0] <= pk["i_kappa"][p] + window and r[1] >= pk["i_kappa"][p] - window:
                    want.append(h)
            assert row.tolist() == want
            if window == 0:
                assert len(row) == pk["votes"][p]
