"""Pins of the oracle's circle fit (CPU only).

The fit is the algebraic least-squares circle through a candidate's hits,
returned as perigee parameters (cos phi0, sin phi0, d0, kappa) with the
turning sign of the peak's kappa bin.  The pins hold it to geometry: exact
circles are recovered, three points give their circumcircle, rotating the
hits rotates phi0 only, the mirrored bin flips every sign, and degenerate
rows are not fitted.
"""

import math

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

G = synth.Grid(64, 8, 64, -10.0, 10.0, -0.0114, 0.0114)


def _kbin(g, kappa):
    return int(math.floor((kappa - g.kappa_min) / ((g.kappa_max - g.kappa_min) / g.n_kappa)))


def _centre_radius(t):
    n = np.array([-t["sin_phi0"], t["cos_phi0"]])
    return (t["d0"] + 1.0 / t["kappa"]) * n, abs(1.0 / t["kappa"])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_exact_helices_are_recovered(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    for _ in range(10):
        phi0 = rng.uniform(0, 2 * math.pi)
        d0 = rng.uniform(-8, 8)
        kap = rng.uniform(0.0015, 0.01) * rng.choice([-1.0, 1.0])
        x, y, _, ok = synth.helix_hits([phi0], [d0], [kap], synth.LAYERS_13)
        x, y = x[0][ok[0]], y[0][ok[0]]
        if x.shape[0] < 5:
            continue
        t = oracle_mod.fit_hits(G, x, y, _kbin(G, kap))
        assert t["status"] == 1 and t["n_hits"] == x.shape[0]
        assert abs(t["cos_phi0"] - math.cos(phi0)) < 1e-5 and abs(t["sin_phi0"] - math.sin(phi0)) < 1e-5
        assert abs(t["d0"] - d0) < 1e-4 * max(1.0, abs(d0)) + 1e-3
        assert abs(t["kappa"] - kap) < 1e-5 * abs(kap)
        assert t["chi2"] < 1e-6 * x.shape[0]


def test_three_points_give_their_circumcircle(oracle_mod):
    """Three non-collinear points: the least-squares circle passes through
    all of them, so it is the circumcircle (centre from the perpendicular
    bisectors, computed here independently)."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        P = rng.uniform(-60, 60, (3, 2)).astype(np.float32).astype(np.float64)
        (ax, ay), (bx, by), (cx, cy) = P
        d = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
        if abs(d) < 1.0:
            continue
        ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / d
        uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / d
        r = math.hypot(ax - ux, ay - uy)
        for k in (5, 50):  # both turning signs describe the same circle
            t = oracle_mod.fit_hits(G, P[:, 0], P[:, 1], k)
            assert t["status"] == 1
            c, R = _centre_radius(t)
            assert abs(c[0] - ux) < 1e-7 * (r + abs(ux)) and abs(c[1] - uy) < 1e-7 * (r + abs(uy))
            assert abs(R - r) < 1e-7 * r
            assert t["chi2"] < 1e-12 * r * r


def test_rotation_turns_phi0_only(oracle_mod):
    phi0, d0, kap = 0.7, -3.0, 0.004
    x, y, _, ok = synth.helix_hits([phi0], [d0], [kap], synth.LAYERS_13)
    x, y = x[0][ok[0]], y[0][ok[0]]
    noise = np.random.default_rng(1).normal(0, 0.01, (2, x.shape[0]))
    x, y = x + noise[0], y + noise[1]
    t0 = oracle_mod.fit_hits(G, x, y, _kbin(G, kap))
    for a in (0.3, 2.0, -1.1):
        xr = x * math.cos(a) - y * math.sin(a)
        yr = x * math.sin(a) + y * math.cos(a)
        t = oracle_mod.fit_hits(G, xr, yr, _kbin(G, kap))
        want = math.atan2(t0["sin_phi0"], t0["cos_phi0"]) + a
        assert abs(t["cos_phi0"] - math.cos(want)) < 1e-5 and abs(t["sin_phi0"] - math.sin(want)) < 1e-5
        assert abs(t["d0"] - t0["d0"]) < 1e-4 and abs(t["kappa"] - t0["kappa"]) < 1e-6 * abs(t0["kappa"])


def test_mirrored_bin_flips_every_sign(oracle_mod):
    """The same hits fitted for a peak in the mirrored kappa bin describe the
    same circle travelled the other way: (phi0 + pi, -d0, -kappa), exactly."""
    rng = np.random.default_rng(4)
    x = rng.uniform(-50, 50, 9)
    y = rng.uniform(-50, 50, 9)
    a = oracle_mod.fit_hits(G, x, y, 10)
    b = oracle_mod.fit_hits(G, x, y, G.n_kappa - 1 - 10)
    assert a["status"] == b["status"] == 1
    for f in ("cos_phi0", "sin_phi0", "d0", "kappa"):
        assert b[f] == -a[f], f
    assert b["chi2"] == a["chi2"]


def test_degenerate_rows_are_not_fitted(oracle_mod):
    rng = np.random.default_rng(9)
    for _ in range(5):  # two points never define a circle (rounding may leave det != 0)
        p = rng.uniform(-40, 40, (2, 2))
        t = oracle_mod.fit_hits(G, p[:, 0], p[:, 1], 5)
        assert t["status"] == 0 and t["n_hits"] == 2
    assert oracle_mod.fit_hits(G, [1.0, 1.0, 1.0], [2.0, 2.0, 2.0], 5)["status"] == 0
    t = oracle_mod.fit_hits(G, [], [], 5)
    assert t["status"] == 0 and t["n_hits"] == 0


def test_fit_of_found_candidates_is_close_to_truth(oracle_mod):
    """On a generated batch event, the fit of the fullest candidate near each
    true track's cell lies close to that track's curvature, although the
    point-vote rows also hold other tracks' hits (a whole-pipeline property,
    so the bound is loose: median within 1.5 kappa bins)."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    g = w.grid
    b = synth.generate(w, n_events=1, first_event=3)
    acc = oracle_mod.vote(g, b.x, b.y, b.event_offsets)
    pk = oracle_mod.peaks(g, acc, w.threshold)
    po, hi = oracle_mod.associate(g, b.x, b.y, b.event_offsets, pk, 1)
    fits = oracle_mod.fit(g, b.x, b.y, pk, po, hi)
    dk = (g.kappa_max - g.kappa_min) / g.n_kappa
    dd = (g.d0_max - g.d0_min) / g.n_d0
    err = []
    for phi0, d0, kap in b.truth_params[0]:
        i = int((phi0 % (2 * math.pi)) / (2 * math.pi / g.n_phi))
        j = int((d0 - g.d0_min) / dd)
        k = int((kap - g.kappa_min) / dk)
        if not (0 <= j < g.n_d0 and 0 <= k < g.n_kappa):
            continue
        di = np.abs(pk["i_phi"] - i)
        di = np.minimum(di, g.n_phi - di)
        sel = np.nonzero((di <= 1) & (np.abs(pk["i_d0"] - j) <= 1) & (np.abs(pk["i_kappa"] - k) <= 1)
                         & (fits["status"] == 1))[0]
        if len(sel) == 0:
            continue
        s = sel[np.argmax(fits["n_hits"][sel])]
        err.append(abs(fits["kappa"][s] - kap) / dk)
    assert len(err) > 100 and np.median(err) < 1.5, (len(err), np.median(err))
