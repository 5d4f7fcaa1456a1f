"""Pins of the oracle's float32 comparison form and of its event-parallel
harness (Section 3's vote, maxima and association; the float32 form is the
one whose disagreement with the binary64 bins is the flip fraction).

* hto_w32 / hto_kbin_fp32 against an independent numpy evaluation in which
  every step is one float32 IEEE operation (np.float32 scalars: no
  contraction, correctly rounded division), on hand-made and random cells.
  An operation-order slip, a swapped product or a fused multiply-add changes
  w in its last bits on a large share of random cells.
* hto_flip_count on a tiny case counted by hand from those two evaluations
  (binary64 bins from the exact-rational-pinned hto_kbin_at), including
  cells whose float32 and binary64 bins differ.
* hto_run_events against the per-event calls on ragged events, with empty
  and one-hit events, at 1, 3 and 16 threads.
"""

import math

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

F = np.float32


def w32_numpy(g, x, y, c, s, d):
    scale = float(g.n_kappa) / (float(F(g.kappa_max)) - float(F(g.kappa_min)))
    S2 = F(2.0 * scale)
    H = F(-float(F(g.kappa_min)) * scale)
    x, y, c, s, d = F(x), F(y), F(c), F(s), F(d)
    r2 = F(F(x * x) + F(y * y))
    q = F(F(y * c) - F(x * s))
    a = F(q - d)
    n = F(a * S2)
    den = F(F(r2 + F(d * d)) - F(F(d + d) * q))
    if not den > F(0.0):
        return math.nan
    v = F(n / den)
    return float(F(v + H))


def kbin32_numpy(g, x, y, c, s, d):
    w = w32_numpy(g, x, y, c, s, d)
    if not (w >= 0.0 and w < float(g.n_kappa)):
        return -1
    return int(w)


def _same(a, b):
    return (math.isnan(a) and math.isnan(b)) or a == b


def test_w32_matches_stepwise_float32(oracle_mod):
    g = synth.Grid(256, 32, 128, -25.0, 25.0, -0.0114, 0.0114)
    c, s, d = oracle_mod.tables(g)
    # hand-made cells: the perigee point (den = 0), a hit on the d0 = 0 line
    # through the origin, far hits, negative coordinates, a straight line
    hand = [(float(-d[3] * s[5]), float(d[3] * c[5]), 5, 3),
            (10.0, 0.0, 0, 16), (-78.0, 3.25, 100, 31), (0.5, -107.9, 200, 0),
            (33.9, 33.9, 64, 15), (-4.4, -0.001, 128, 17)]
    for x, y, i, j in hand:
        a = oracle_mod.w32(g, x, y, c[i], s[i], d[j])
        b = w32_numpy(g, x, y, c[i], s[i], d[j])
        assert _same(a, b), (x, y, i, j, a, b)
    rng = np.random.default_rng(7)
    n = 4000
    r = rng.choice(synth.LAYERS_13, n)
    th = rng.uniform(0, 2 * np.pi, n)
    xs, ys = (r * np.cos(th)).astype(np.float32), (r * np.sin(th)).astype(np.float32)
    ii, jj = rng.integers(0, g.n_phi, n), rng.integers(0, g.n_d0, n)
    for t in range(n):
        a = oracle_mod.w32(g, xs[t], ys[t], c[ii[t]], s[ii[t]], d[jj[t]])
        b = w32_numpy(g, xs[t], ys[t], c[ii[t]], s[ii[t]], d[jj[t]])
        assert _same(a, b), (t, a, b)
        assert oracle_mod.kbin_fp32(g, xs[t], ys[t], c[ii[t]], s[ii[t]], d[jj[t]]) == \
            kbin32_numpy(g, xs[t], ys[t], c[ii[t]], s[ii[t]], d[jj[t]])


def test_w32_stepwise_model_detects_contraction():
    """The numpy model itself tells the fused and unfused forms apart on
    random cells: a contraction on either side would be caught above."""
    g = synth.Grid(256, 32, 128, -25.0, 25.0, -0.0114, 0.0114)
    rng = np.random.default_rng(3)
    differ = 0
    for _ in range(2000):
        x, y = F(rng.uniform(-100, 100)), F(rng.uniform(-100, 100))
        c, s = F(math.cos(rng.uniform(0, 6.3))), F(math.sin(rng.uniform(0, 6.3)))
        q_sep = F(F(y * c) - F(x * s))
        q_fma = F(float(y) * float(c) - float(F(x * s)))  # one rounding of y*c - fl(x*s)
        differ += q_sep != q_fma
    assert differ > 100


def _edge_hits(g, c, s, d, i, j, n, rng):
    """Hits on circles of cell column (i, j) whose binary64 w lies within a
    few 1e-6 bins of a bin edge (seeded): where the float32 form can flip."""
    phi = math.atan2(float(s[i]), float(c[i]))
    d0 = float(d[j])
    dk = (g.kappa_max - g.kappa_min) / g.n_kappa
    out = []
    for _ in range(n):
        k = int(rng.integers(1, g.n_kappa))
        if 2 * k == g.n_kappa:  # kappa = 0: a straight line, not a circle
            continue
        kap = g.kappa_min + k * dk
        r = float(rng.choice(synth.LAYERS_13))
        x, y, _, ok = synth.helix_hits([phi], [d0], [kap], [r])
        if ok[0, 0] and np.isfinite(x[0, 0]) and np.isfinite(y[0, 0]):
            out.append((F(x[0, 0]), F(y[0, 0])))
    return out


def test_flip_count_tiny_case_by_hand(oracle_mod):
    g = synth.Grid(16, 4, 32, -10.0, 10.0, -0.0114, 0.0114)
    c, s, d = oracle_mod.tables(g)
    rng = np.random.default_rng(11)
    cand = _edge_hits(g, c, s, d, 5, 2, 400, rng)
    flips = []
    for x, y in cand:
        if oracle_mod.kbin_at(g, x, y, c[5], s[5], d[2]) != kbin32_numpy(g, x, y, c[5], s[5], d[2]):
            flips.append((x, y))
        if len(flips) == 2:
            break
    assert len(flips) == 2
    plain = [(F(30.0), F(-12.5)), (F(-4.4), F(0.25)), (F(60.8), F(60.8))]
    hits = flips + plain
    v64 = v32 = diff = 0
    for x, y in hits:
        for i in range(g.n_phi):
            for j in range(g.n_d0):
                k64 = oracle_mod.kbin_at(g, x, y, c[i], s[i], d[j])
                k32 = kbin32_numpy(g, x, y, c[i], s[i], d[j])
                v64 += k64 >= 0
                v32 += k32 >= 0
                diff += k64 != k32
    xs = np.array([h[0] for h in hits], np.float32)
    ys = np.array([h[1] for h in hits], np.float32)
    assert diff >= 2 and v64 > 30
    assert oracle_mod.flip_count(g, xs, ys) == (v64, v32, diff)
    # two events: the counts add up over event boundaries
    offs = np.array([0, 2, 5], np.int32)
    assert oracle_mod.flip_count(g, xs, ys, offs) == (v64, v32, diff)


def _per_event(oracle_mod, g, b, thr, window):
    votes = peaks = pairs = 0
    for e in range(b.n_events):
        be = b.event(e)
        acc = oracle_mod.vote(g, be.x, be.y)
        votes += int(acc.sum(dtype=np.int64))
        pk = oracle_mod.peaks(g, acc, thr)
        peaks += len(pk)
        _, hi = oracle_mod.associate(g, be.x, be.y, None, pk, window)
        pairs += len(hi)
    return votes, peaks, pairs


def test_run_events_equals_per_event_calls(oracle_mod):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    g = synth.Grid(32, 8, 32, -25.0, 25.0, -0.0114, 0.0114)
    b = synth.generate(w, n_events=6)
    # ragged: insert an empty event and a one-hit event
    xs = [b.event(e).x for e in range(6)]
    ys = [b.event(e).y for e in range(6)]
    xs.insert(2, np.zeros(0, np.float32))
    ys.insert(2, np.zeros(0, np.float32))
    xs.insert(5, xs[0][:1].copy())
    ys.insert(5, ys[0][:1].copy())
    offs = np.concatenate([[0], np.cumsum([len(v) for v in xs])]).astype(np.int32)
    bb = synth.from_arrays(np.concatenate(xs), np.concatenate(ys), event_offsets=offs)
    assert bb.n_events == 8
    want = _per_event(oracle_mod, g, bb, 5, 1)
    assert want[0] > 0 and want[1] > 0 and want[2] > 0
    for threads in (1, 3, 16):
        assert oracle_mod.run_events(g, bb.x, bb.y, bb.event_offsets, 5, 1, threads) == want
    # window 0 and another threshold change the pair and peak totals consistently
    assert oracle_mod.run_events(g, bb.x, bb.y, bb.event_offsets, 7, 0, 4) == _per_event(oracle_mod, g, bb, 7, 0)
