"""Pins of the oracle's straight-line vote (the paper's kappa = 0 model, CPU only).

On a grid with one kappa bin, each hit votes in every phi0 row for the d0
bin of q = y cos phi0 - x sin phi0.  The pins: a straight track through a
row's centre direction puts every hit in one d0 bin, the bins equal an exact
rational evaluation (away from bin edges), and association rows hold the
hits whose bin lies within the window.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

G = synth.Grid(256, 64, 1, -40.0, 40.0, -0.0005, 0.0005)


@pytest.mark.parametrize("seed", [0, 1])
def test_bin_centre_line_puts_every_hit_in_its_cell(oracle_mod, seed):
    c, s, d = oracle_mod.tables(G)
    rng = np.random.default_rng(seed)
    for _ in range(10):
        i = int(rng.integers(0, G.n_phi))
        j = int(rng.integers(4, G.n_d0 - 4))
        phi0 = math.atan2(float(s[i]), float(c[i]))
        d0 = float(d[j])
        x, y, _, ok = synth.helix_hits([phi0], [d0], [1e-9], synth.LAYERS_13)
        hx, hy = x[0][ok[0]].astype(np.float32), y[0][ok[0]].astype(np.float32)
        acc = oracle_mod.vote_line(G, hx, hy)[0, :, :, 0]
        assert acc[i, j] == hx.shape[0], (i, j, acc[i, j], hx.shape[0])
        assert acc[i].sum() == hx.shape[0]   # one vote per hit in each row


def test_line_bins_equal_exact_rational_evaluation(oracle_mod):
    """Rational q = y c - x s of the float inputs and its bin; the binary64
    bin must agree wherever q is not within 1e-9 of a bin edge."""
    c, s, d = oracle_mod.tables(G)
    rng = np.random.default_rng(4)
    x = rng.uniform(-100, 100, 60).astype(np.float32)
    y = rng.uniform(-100, 100, 60).astype(np.float32)
    width = Fraction(float(np.float32(G.d0_max))) - Fraction(float(np.float32(G.d0_min)))
    checked = 0
    for h in range(60):
        for i in range(0, G.n_phi, 7):
            q = Fraction(float(y[h])) * Fraction(float(c[i])) - Fraction(float(x[h])) * Fraction(float(s[i]))
            t = (q - Fraction(float(np.float32(G.d0_min)))) * G.n_d0 / width
            k = oracle_mod.line_bin(G, x[h], y[h], i)
            if abs(t - round(t)) < Fraction(1, 10 ** 9):
                continue
            want = math.floor(t) if 0 <= t < G.n_d0 else -1
            assert k == want, (h, i)
            checked += 1
    assert checked > 1500


def test_line_association_rows(oracle_mod):
    rng = np.random.default_rng(2)
    phi0 = rng.uniform(0, 2 * math.pi, 12)
    d0 = rng.uniform(-30, 30, 12)
    x, y, _, ok = synth.helix_hits(phi0, d0, np.full(12, 1e-9), synth.LAYERS_13)
    hx, hy = x[ok].astype(np.float32), y[ok].astype(np.float32)
    acc = oracle_mod.vote_line(G, hx, hy)
    pk = oracle_mod.peaks(G, acc, 8)
    assert len(pk) >= 12
    for window in (0, 1, 2):
        po, hi = oracle_mod.associate_line(G, hx, hy, None, pk, window)
        for p in range(len(pk)):
            row = hi[po[p]:po[p + 1]]
            want = [h for h in range(hx.shape[0])
                    if (jh := oracle_mod.line_bin(G, hx[h], hy[h], pk["i_phi"][p])) >= 0
                    and abs(jh - pk["i_d0"][p]) <= window]
            assert row.tolist() == want
            if window == 0:
                assert len(row) == pk["votes"][p]
