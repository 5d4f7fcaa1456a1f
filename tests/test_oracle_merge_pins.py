"""Pins of the oracle's duplicate and mirror merging (CPU only).

After the circle fit a candidate is UNFITTED (fit status != 1), BACKWARD (its
hits do not lie ahead of its perigee along (cos phi0, sin phi0)), a
DUPLICATE (a better forward fitted candidate of its event lies within the
radius in phi0 (periodic), d0 and kappa; better = more votes, then smaller
index) or KEPT.  The pins: a hand-worked case whose states are derived below
for four radii, mirror pairs of exact tracks, nesting of the kept sets over
radii, and that merging keeps the tracks the candidates found.
"""

import math

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

K, D, B, U = 1, 0, -1, -2   # kept, duplicate, backward, unfitted
HG = synth.Grid(8, 6, 6, -3.0, 3.0, -0.01, 0.01)


def _hand_case(oracle_mod):
    """Two events on an 8 x 6 x 6 grid.  Event 0 holds hits 0..29 at
    (10 + h, -5); event 1 holds hits 30..55 at (20 - h, 20).  Event 0's fits
    point along +x (cos 1, sin 0), so h.t = x > 0; event 1's along +y, so
    h.t = y > 0 although x < 0.  Each candidate's row is 5 hits of its event.

    idx    ev (i, j, k)  votes  fit
     0 A   0  (0, 2, 2)   10
     1 B   0  (7, 2, 3)   12    phi0 distance to A is 1 (periodic)
     2 C   0  (2, 2, 2)   11    distance 2 to A, 3 to B
     3 D   0  (4, 4, 4)    9    distance 2 to C in every index
     4 E   0  (5, 5, 5)    9    distance 1 to D, as many votes, later index
     5 F   0  (1, 2, 2)   20    points along -x: backward
     6 G   0  (3, 2, 2)   30    status 0: unfitted
     7 H   1  (0, 2, 2)    5    A's cell, other event
     8 I   1  (4, 0, 0)    7
     9 J   1  (4, 0, 3)    7    distance 3 to I, later index

    radius 2: A dup (B); B kept; C kept (A is worse, B too far, F and G do
      not count); D dup (C); E dup (D, although D is itself a duplicate);
      H, I, J kept.
    radius 1: A dup (B); C kept; D kept (E is not better); E dup (D).
    radius 0: every forward fitted candidate kept.
    radius 3: C dup (B: distance 3, 1 in kappa, more votes); J dup (I).
    """
    x = np.zeros(56, np.float32)
    y = np.zeros(56, np.float32)
    x[:30] = 10 + np.arange(30)
    y[:30] = -5
    x[30:] = 20 - np.arange(30, 56)
    y[30:] = 20
    cells = [(0, 0, 2, 2, 10), (0, 7, 2, 3, 12), (0, 2, 2, 2, 11), (0, 4, 4, 4, 9), (0, 5, 5, 5, 9),
             (0, 1, 2, 2, 20), (0, 3, 2, 2, 30), (1, 0, 2, 2, 5), (1, 4, 0, 0, 7), (1, 4, 0, 3, 7)]
    pk = np.array(cells, oracle_mod.PEAK_DTYPE)
    rows = [np.arange(5 * c, 5 * c + 5) if c < 7 else np.arange(30 + 5 * (c - 7), 35 + 5 * (c - 7))
            for c in range(10)]
    po = np.zeros(11, np.int64)
    po[1:] = np.cumsum([len(r) for r in rows])
    hi = np.concatenate(rows).astype(np.int32)
    fits = np.zeros(10, oracle_mod.TRACK_DTYPE)
    fits["status"] = 1
    fits["status"][6] = 0
    fits["n_hits"] = 5
    fits["chi2"] = 1.0
    fits["cos_phi0"] = [1.0] * 7 + [0.0] * 3
    fits["sin_phi0"] = [0.0] * 7 + [1.0] * 3
    fits["cos_phi0"][5] = -1.0
    return x, y, pk, po, hi, fits


HAND = {
    2: [D, K, K, D, D, B, U, K, K, K],
    1: [D, K, K, K, D, B, U, K, K, K],
    0: [K, K, K, K, K, B, U, K, K, K],
    3: [D, K, D, D, D, B, U, K, K, D],
}


@pytest.mark.parametrize("radius", sorted(HAND))
def test_hand_worked_states(oracle_mod, radius):
    x, y, pk, po, hi, fits = _hand_case(oracle_mod)
    state, kept = oracle_mod.merge(HG, x, y, pk, po, hi, fits, radius)
    assert state.tolist() == HAND[radius]
    assert kept == HAND[radius].count(K)


def test_mirror_pairs_of_exact_tracks(oracle_mod):
    """Unsmeared tracks at bin centres give a peak at their cell and one at
    the mirror cell (phi0 + pi, -d0, -kappa).  After merging, each track
    keeps a forward candidate along its direction, and every fitted
    candidate pointing against a track is backward."""
    g = synth.WORKLOADS["single_event_10trk"].grid
    c, s, d = oracle_mod.tables(g)
    dk = (g.kappa_max - g.kappa_min) / g.n_kappa
    rng = np.random.default_rng(6)
    rows_i = rng.choice(g.n_phi // 2, 6, replace=False)   # directions within one half-turn: none opposite
    truth = []
    xs, ys = [], []
    for i in rows_i:
        j = int(rng.integers(1, g.n_d0 - 1))
        k = int(rng.choice([int(rng.integers(8, 26)), int(rng.integers(38, 56))]))
        phi0 = math.atan2(float(s[i]), float(c[i]))
        kap = g.kappa_min + (k + 0.5) * dk
        x, y, _, ok = synth.helix_hits([phi0], [float(d[j])], [kap], synth.LAYERS_13)
        xs.append(x[0][ok[0]])
        ys.append(y[0][ok[0]])
        truth.append(phi0)
    hx = np.concatenate(xs).astype(np.float32)
    hy = np.concatenate(ys).astype(np.float32)
    acc = oracle_mod.vote(g, hx, hy)
    pk = oracle_mod.peaks(g, acc, 8)
    po, hi = oracle_mod.associate(g, hx, hy, None, pk, 0)
    fits = oracle_mod.fit(g, hx, hy, pk, po, hi)
    state, kept = oracle_mod.merge(g, hx, hy, pk, po, hi, fits, 2)
    fitted = fits["status"] == 1
    assert np.all(state[fitted] != U) and np.all(state[~fitted] == U)
    direction = np.arctan2(fits["sin_phi0"], fits["cos_phi0"])
    for phi0 in truth:
        gap = np.abs((direction - phi0 + math.pi) % (2 * math.pi) - math.pi)
        along = fitted & (gap < 0.1)
        against = fitted & (gap > math.pi - 0.1)
        assert along.any() and against.any()
        assert np.all(state[against] == B), phi0
        assert np.any(state[along] == K), phi0
    assert kept >= len(truth)


def _batch_candidates(oracle_mod, first_event, n_events=1):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    g = w.grid
    b = synth.generate(w, n_events=n_events, first_event=first_event)
    acc = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk = oracle_mod.peaks(g, acc, w.threshold)
    po, hi = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk, 1)
    fits = oracle_mod.fit(g, b.x, b.y, pk, po, hi)
    return g, b, pk, po, hi, fits


def test_kept_sets_nest_over_radii(oracle_mod):
    """Radius 0 keeps every forward fitted candidate (no two peaks share a
    cell), and so does radius 1: by the peak rule no two peaks are
    neighbours.  A larger radius keeps a strict subset; mirrors and fit
    status do not depend on the radius."""
    g, b, pk, po, hi, fits = _batch_candidates(oracle_mod, 1)
    states = [oracle_mod.merge(g, b.x, b.y, pk, po, hi, fits, r)[0] for r in range(4)]
    assert np.all(states[0] != D)
    assert np.array_equal(states[1], states[0])
    for r in range(2, 4):
        assert np.array_equal(states[r] < 0, states[0] < 0)
        assert np.array_equal(states[r][states[r] < 0], states[0][states[0] < 0])
        assert np.all(states[r - 1][states[r] == K] == K)
        assert (states[r] == K).sum() < (states[r - 1] == K).sum()


def test_merging_keeps_the_found_tracks(oracle_mod):
    """On a generated batch event, a true track counts as found by a set of
    candidates when one of them holds at least 5 of its hits, more than of
    any other track.  The kept candidates (radius 2) find at least 95 % of
    the tracks that all fitted candidates find, with at most 30 % of them."""
    g, b, pk, po, hi, fits = _batch_candidates(oracle_mod, 0)
    state, kept = oracle_mod.merge(g, b.x, b.y, pk, po, hi, fits, 2)

    def found(sel):
        out = set()
        for p in np.nonzero(sel)[0]:
            t = b.truth_track[hi[po[p]:po[p + 1]]]
            t = t[t >= 0]
            if t.size == 0:
                continue
            v, n = np.unique(t, return_counts=True)
            a = np.argmax(n)
            if n[a] >= 5:
                out.add(int(v[a]))
        return out

    before = found(fits["status"] == 1)
    after = found(state == K)
    assert len(before) > 100
    assert after <= before and len(after) >= 0.95 * len(before), (len(after), len(before))
    assert kept <= 0.3 * (fits["status"] == 1).sum(), (kept, (fits["status"] == 1).sum())
