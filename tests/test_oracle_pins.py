"""Pins of the CPU oracle against facts the method and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
closed form, a textbook special case, exact rational arithmetic, a
hand-derived answer or an invariant (Section 3 of the paper defines the
transform; its two 2-parameter models are the d0 = 0 and kappa = 0 cases).
"""

import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _grid(n_phi, n_d0, n_kappa, d0_min, d0_max, k_min, k_max):
    return synth.Grid(n_phi, n_d0, n_kappa, d0_min, d0_max, k_min, k_max)


# ---------------------------------------------------------------- tables

def test_tables_are_bin_centres(oracle_mod):
    g = _grid(12, 5, 8, -10.0, 15.0, -0.01, 0.01)
    c, s, d = oracle_mod.tables(g)
    phi = np.arctan2(s.astype(np.float64), c.astype(np.float64)) % (2 * math.pi)
    # phi_i = (i + 1/2) * 2pi / n_phi, to float32 accuracy of cos/sin
    assert np.allclose(phi, (np.arange(12) + 0.5) * 2 * math.pi / 12, atol=1e-6)
    assert np.allclose(c.astype(np.float64) ** 2 + s.astype(np.float64) ** 2, 1.0, atol=1e-6)
    # d0 centres: -7.5, -2.5, 2.5, 7.5, 12.5 exactly representable
    assert d.tolist() == [-7.5, -2.5, 2.5, 7.5, 12.5]


# ---------------------------------------------------------------- closed form

def _centre(g, i, j, k):
    phi0 = (i + 0.5) * 2 * math.pi / g.n_phi
    d0 = g.d0_min + (j + 0.5) * (g.d0_max - g.d0_min) / g.n_d0
    kap = float(np.float32(g.kappa_min)) + (k + 0.5) * (float(np.float32(g.kappa_max)) - float(np.float32(g.kappa_min))) / g.n_kappa
    return phi0, d0, kap


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bin_centre_helix_votes_into_its_cell_and_mirror(oracle_mod, seed):
    """A track generated exactly on a bin-centre helix puts every hit in that
    cell, and (phi0 + pi, -d0, -kappa), the same circle, in the mirror cell."""
    g = _grid(64, 8, 64, -10.0, 10.0, -0.0114, 0.0114)
    rng = np.random.default_rng(seed)
    for _ in range(4):
        i, j, k = int(rng.integers(0, 64)), int(rng.integers(0, 8)), int(rng.integers(8, 56))
        phi0, d0, kap = _centre(g, i, j, k)
        x, y, _, ok = synth.helix_hits([phi0], [d0], [kap], synth.LAYERS_13)
        x = x[ok].astype(np.float32)
        y = y[ok].astype(np.float32)
        n = x.shape[0]
        assert n >= 8
        acc = oracle_mod.vote(g, x, y)[0]
        assert acc[i, j, k] == n
        assert acc[(i + 32) % 64, 7 - j, 63 - k] == n
        assert acc.max() == n


# ---------------------------------------------------------------- textbook reductions

def test_d0_zero_reduces_to_circle_through_origin(oracle_mod):
    """n_d0 = 1 on a symmetric range puts the only d0 centre at 0, where the
    vote must equal the 2-parameter origin model kappa = 2 q / r^2."""
    g = _grid(48, 1, 40, -1.0, 1.0, -0.02, 0.02)
    c, s, d = oracle_mod.tables(g)
    assert d[0] == 0.0
    rng = np.random.default_rng(5)
    r = rng.uniform(5.0, 100.0, 300)
    ph = rng.uniform(0, 2 * math.pi, 300)
    x = (r * np.cos(ph)).astype(np.float32)
    y = (r * np.sin(ph)).astype(np.float32)
    acc = oracle_mod.vote(g, x, y)[0]
    X, Y = x.astype(np.float64)[:, None], y.astype(np.float64)[:, None]
    C, S = c.astype(np.float64)[None, :], s.astype(np.float64)[None, :]
    kap = 2.0 * (Y * C - X * S) / (X * X + Y * Y)
    kmin, kmax = float(np.float32(-0.02)), float(np.float32(0.02))
    w = (kap - kmin) * 40 / (kmax - kmin)
    ref = np.zeros((48, 1, 40), np.uint32)
    hh, ii = np.nonzero((w >= 0) & (w < 40))
    np.add.at(ref, (ii, 0, np.floor(w[hh, ii]).astype(int)), 1)
    assert ref.sum() > 1000
    assert np.array_equal(acc, ref)


def test_kappa_zero_reduces_to_straight_line_transform(oracle_mod):
    """With n_kappa = 2 over a huge symmetric kappa range, bin 1 holds exactly
    the hits with q >= d0_j, so the differences along d0 are the straight-line
    (normal form) Hough transform of the paper's displaced-track model."""
    g = _grid(30, 24, 2, -12.0, 12.0, -1.0e4, 1.0e4)
    c, s, d = oracle_mod.tables(g)
    rng = np.random.default_rng(11)
    r = rng.uniform(25.0, 100.0, 400)
    ph = rng.uniform(0, 2 * math.pi, 400)
    x = (r * np.cos(ph)).astype(np.float32)
    y = (r * np.sin(ph)).astype(np.float32)
    acc = oracle_mod.vote(g, x, y)[0].astype(np.int64)
    assert np.all(acc.sum(axis=2) == 400)  # every hit votes in every column
    rho = y.astype(np.float64)[:, None] * c.astype(np.float64)[None, :] - \
        x.astype(np.float64)[:, None] * s.astype(np.float64)[None, :]          # [hit, phi]
    for i in range(30):
        ge = (rho[:, i][:, None] >= d.astype(np.float64)[None, :]).sum(axis=0)
        assert np.array_equal(acc[i, :, 1], ge)
        hist, _ = np.histogram(rho[:, i], bins=d.astype(np.float64))
        assert np.array_equal(acc[i, :-1, 1] - acc[i, 1:, 1], hist)


# ---------------------------------------------------------------- exact rational brute force

def _exact_bin(g, x, y, c, s, d):
    X, Y, C, S, D = (Fraction(float(v)) for v in (x, y, c, s, d))
    q = Y * C - X * S
    den = X * X + Y * Y + D * D - 2 * D * q
    if den <= 0:
        return -1
    kap = 2 * (q - D) / den
    kmin = Fraction(float(np.float32(g.kappa_min)))
    kmax = Fraction(float(np.float32(g.kappa_max)))
    w = (kap - kmin) * g.n_kappa / (kmax - kmin)
    if w < 0 or w >= g.n_kappa:
        return -1
    return math.floor(w)


@pytest.mark.parametrize("seed", [0, 1])
def test_vote_equals_exact_rational_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    g = _grid(7, 5, 9, -6.0, 9.0, -0.08, 0.05)
    c, s, d = oracle_mod.tables(g)
    r = rng.uniform(3.0, 40.0, 16)
    ph = rng.uniform(0, 2 * math.pi, 16)
    x = (r * np.cos(ph)).astype(np.float32)
    y = (r * np.sin(ph)).astype(np.float32)
    ref = np.zeros((7, 5, 9), np.uint32)
    for h in range(16):
        for i in range(7):
            for j in range(5):
                k = _exact_bin(g, x[h], y[h], c[i], s[i], d[j])
                if k >= 0:
                    ref[i, j, k] += 1
    assert ref.sum() > 50
    assert np.array_equal(oracle_mod.vote(g, x, y)[0], ref)


def test_perigee_hit_casts_no_vote(oracle_mod):
    """den = |h - P|^2 = 0 when the hit is the perigee point itself."""
    g = _grid(8, 4, 16, -8.0, 8.0, -0.05, 0.05)
    c, s, d = oracle_mod.tables(g)
    # P = d0 * n, n = (-sin, cos); choose values whose products are exact
    i, j = 0, 3
    px, py = float(np.float32(-d[j] * np.float64(s[i]))), float(np.float32(d[j] * np.float64(c[i])))
    w = oracle_mod.w64(g, px, py, c[i], s[i], d[j])
    assert math.isnan(w) or oracle_mod.kbin_at(g, px, py, c[i], s[i], d[j]) == _exact_bin(g, px, py, c[i], s[i], d[j])
    # a hit exactly on the d0 = 0 perigee (the origin) never votes in d0 = 0 columns
    g0 = _grid(8, 1, 16, -1.0, 1.0, -0.05, 0.05)
    assert all(oracle_mod.kbin(g0, 0.0, 0.0, i, 0) == -1 for i in range(8))


def test_bin_edges_are_half_open(oracle_mod):
    """kappa exactly on a bin edge belongs to the upper bin; w = n_kappa is out."""
    # symmetric grid, d0 = 0 column: kappa = 2 y / r^2 for a hit on the y axis (phi0 = pi/2 -> c = 0?)
    g = _grid(4, 1, 4, -1.0, 1.0, -0.5, 0.5)
    # hit (0, y): with phi_i the column centre, kappa = 2 (y c) / y^2 = 2 c / y
    c, s, d = oracle_mod.tables(g)
    for i in range(4):
        for yv in (4.0, 8.0, -4.0, 2.0):
            k = oracle_mod.kbin_at(g, 0.0, yv, c[i], s[i], d[0])
            assert k == _exact_bin(g, 0.0, yv, c[i], s[i], d[0])
    # exact edge: kappa = 0 -> w = 2 exactly -> bin 2 (upper), for a hit with q = 0
    assert oracle_mod.kbin_at(g, 3.0, 0.0, 1.0, 0.0, 0.0) == 2
    # kappa = kappa_max exactly is out of range: q = 1/4 * r^2 ... hit (0, 4), c = 1: kappa = 2*4/16 = 0.5
    assert oracle_mod.kbin_at(g, 0.0, 4.0, 1.0, 0.0, 0.0) == -1
    # kappa = kappa_min exactly is bin 0: hit (0, -4), c = 1: kappa = -0.5
    assert oracle_mod.kbin_at(g, 0.0, -4.0, 1.0, 0.0, 0.0) == 0


# ---------------------------------------------------------------- peak rule (hand-derived)

def _acc(shape, cells):
    a = np.zeros(shape, np.uint32)
    for (i, j, k), v in cells.items():
        a[i, j, k] = v
    return a[None]


def test_peak_plateau_keeps_lowest_linear_index(oracle_mod):
    g = _grid(6, 5, 7, -1.0, 1.0, -1.0, 1.0)
    acc = _acc((6, 5, 7), {(2, 2, 3): 10, (2, 2, 4): 10, (2, 3, 3): 10, (3, 1, 1): 4})
    pk = oracle_mod.peaks(g, acc, 5)
    assert [(p["i_phi"], p["i_d0"], p["i_kappa"], p["votes"]) for p in pk] == [(2, 2, 3, 10)]


def test_peak_threshold_and_strictness(oracle_mod):
    g = _grid(6, 5, 7, -1.0, 1.0, -1.0, 1.0)
    acc = _acc((6, 5, 7), {(1, 1, 1): 8, (4, 3, 5): 7, (4, 3, 4): 6})
    got = [(p["i_phi"], p["i_d0"], p["i_kappa"]) for p in oracle_mod.peaks(g, acc, 8)]
    assert got == [(1, 1, 1)]
    got = [(p["i_phi"], p["i_d0"], p["i_kappa"]) for p in oracle_mod.peaks(g, acc, 7)]
    assert got == [(1, 1, 1), (4, 3, 5)]


def test_peak_phi_wraps_but_d0_kappa_do_not(oracle_mod):
    g = _grid(6, 5, 7, -1.0, 1.0, -1.0, 1.0)
    # (0, 2, 3) = 9 next to (5, 2, 3) = 10 across the phi wrap: only (5, 2, 3) is a peak
    acc = _acc((6, 5, 7), {(0, 2, 3): 9, (5, 2, 3): 10})
    got = [(p["i_phi"], p["i_d0"], p["i_kappa"]) for p in oracle_mod.peaks(g, acc, 1)]
    assert got == [(5, 2, 3)]
    # equal across the wrap: (0, ...) has the lower linear index and wins
    acc = _acc((6, 5, 7), {(0, 2, 3): 10, (5, 2, 3): 10})
    got = [(p["i_phi"], p["i_d0"], p["i_kappa"]) for p in oracle_mod.peaks(g, acc, 1)]
    assert got == [(0, 2, 3)]
    # corners of d0 / kappa have no outside neighbours
    acc = _acc((6, 5, 7), {(3, 0, 0): 5, (3, 4, 6): 5})
    got = [(p["i_phi"], p["i_d0"], p["i_kappa"]) for p in oracle_mod.peaks(g, acc, 1)]
    assert got == [(3, 0, 0), (3, 4, 6)]


def test_peak_rule_small_phi_counts(oracle_mod):
    """n_phi = 1 and 2: a neighbour reached both ways is the same cell."""
    g1 = _grid(1, 3, 3, -1.0, 1.0, -1.0, 1.0)
    acc = _acc((1, 3, 3), {(0, 1, 1): 3})
    assert [(p["i_d0"], p["i_kappa"]) for p in oracle_mod.peaks(g1, acc, 1)] == [(1, 1)]
    g2 = _grid(2, 3, 3, -1.0, 1.0, -1.0, 1.0)
    acc = _acc((2, 3, 3), {(0, 1, 1): 3, (1, 1, 1): 3})
    assert [(p["i_phi"], p["i_d0"], p["i_kappa"]) for p in oracle_mod.peaks(g2, acc, 1)] == [(0, 1, 1)]


def test_no_two_adjacent_peaks_random(oracle_mod):
    """The tie rule never marks two neighbouring cells (random plateaus)."""
    g = _grid(9, 6, 8, -1.0, 1.0, -1.0, 1.0)
    rng = np.random.default_rng(3)
    acc = rng.integers(0, 3, (1, 9, 6, 8)).astype(np.uint32)
    pk = oracle_mod.peaks(g, acc, 1)
    cells = {(int(p["i_phi"]), int(p["i_d0"]), int(p["i_kappa"])) for p in pk}
    assert cells
    for (i, j, k) in cells:
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for dk in (-1, 0, 1):
                    if (di, dj, dk) != (0, 0, 0):
                        assert ((i + di) % 9, j + dj, k + dk) not in cells
    # and every 3x3x3 neighbourhood maximum at or above threshold that is unique is a peak
    for i in range(9):
        for j in range(1, 5):
            for k in range(1, 7):
                v = acc[0, i, j, k]
                nb = [acc[0, (i + di) % 9, j + dj, k + dk] for di in (-1, 0, 1) for dj in (-1, 0, 1)
                      for dk in (-1, 0, 1) if (di, dj, dk) != (0, 0, 0)]
                if v >= 1 and v > max(nb):
                    assert (i, j, k) in cells


# ---------------------------------------------------------------- association

def test_association_window_and_order(oracle_mod):
    g = _grid(16, 4, 32, -10.0, 10.0, -0.02, 0.02)
    c, s, d = oracle_mod.tables(g)
    rng = np.random.default_rng(8)
    r = rng.uniform(5.0, 100.0, 60)
    ph = rng.uniform(0, 2 * math.pi, 60)
    x = (r * np.cos(ph)).astype(np.float32)
    y = (r * np.sin(ph)).astype(np.float32)
    offs = np.array([0, 25, 25, 60], np.int32)  # middle event empty
    acc = oracle_mod.vote(g, x, y, offs)
    pk = oracle_mod.peaks(g, acc, 2)
    assert len(pk) > 0 and set(pk["event"].tolist()) <= {0, 2}
    po, hi = oracle_mod.associate(g, x, y, offs, pk, 1)
    for p in range(len(pk)):
        e, i, j, k = (int(pk[p][f]) for f in ("event", "i_phi", "i_d0", "i_kappa"))
        members = hi[po[p]:po[p + 1]]
        assert np.all(np.diff(members) > 0)
        assert np.all((members >= offs[e]) & (members < offs[e + 1]))
        # count = votes of the window cells (each hit votes once per column)
        assert len(members) == int(acc[e, i, j, max(0, k - 1):k + 2].sum())
        for h in members:
            assert abs(_exact_bin(g, x[h], y[h], c[i], s[i], d[j]) - k) <= 1


# ---------------------------------------------------------------- invariants

def test_total_votes_equals_in_range_columns(oracle_mod):
    w = synth.WORKLOADS["single_event_10trk"]
    b = synth.generate(w)
    g = w.grid
    c, s, d = oracle_mod.tables(g)
    acc = oracle_mod.vote(g, b.x, b.y)[0]
    X, Y = b.x.astype(np.float64)[:, None, None], b.y.astype(np.float64)[:, None, None]
    C, S = c.astype(np.float64)[None, :, None], s.astype(np.float64)[None, :, None]
    D = d.astype(np.float64)[None, None, :]
    q = Y * C - X * S
    kap = 2 * (q - D) / (X * X + Y * Y + D * D - 2 * D * q)
    kmin, kmax = float(np.float32(g.kappa_min)), float(np.float32(g.kappa_max))
    wv = (kap - kmin) * g.n_kappa / (kmax - kmin)
    assert int(acc.sum()) == int(((wv >= 0) & (wv < g.n_kappa)).sum())


def test_mirror_symmetry_and_permutation_invariance(oracle_mod):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=1, first_event=13)
    g = synth.Grid(64, 16, 32, -25.0, 25.0, -0.0114, 0.0114)
    acc = oracle_mod.vote(g, b.x, b.y)[0]
    mirror = acc[np.r_[32:64, 0:32]][:, ::-1, ::-1]
    assert (acc != mirror).sum() <= 2
    perm = np.random.default_rng(0).permutation(b.n_hits)
    acc_p = oracle_mod.vote(g, b.x[perm], b.y[perm])[0]
    assert np.array_equal(acc, acc_p)
    pk = oracle_mod.peaks(g, acc[None], 6)
    assert np.array_equal(pk, oracle_mod.peaks(g, acc_p[None], 6))


def test_batched_equals_per_event(oracle_mod):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    g = synth.Grid(32, 8, 16, -25.0, 25.0, -0.0114, 0.0114)
    b = synth.generate(w, n_events=3)
    acc = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    for e in range(3):
        be = b.event(e)
        assert np.array_equal(acc[e], oracle_mod.vote(g, be.x, be.y)[0])


def test_fp32_op_order_flip_fraction_is_reported_small(oracle_mod):
    """The plain float32 op order disagrees with the binary64 bins on a small
    fraction of columns (the reason the bin is defined in binary64)."""
    w = synth.WORKLOADS["dense_event_500trk"]
    b = synth.generate(w)
    sel = np.random.default_rng(1).choice(b.n_hits, 300, replace=False)
    v64, v32, diff = oracle_mod.flip_count(w.grid, b.x[sel], b.y[sel])
    assert v64 > 1_000_000 and abs(v64 - v32) <= diff
    assert diff / v64 < 1e-3
