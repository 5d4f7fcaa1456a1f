"""Pins of the oracle's second Hough transform (displaced vertices, CPU only).

Every candidate (phi_i, d0_j) votes along its line y cos(phi_i) - x sin(phi_i)
= d0_j in an (x, y) grid, walking the less steep axis; vertices are the 2-D
local maxima.  The pins hold it to geometry: lines through one point meet in
that point's cell, each vote lies on its line, the peak rule is the first
transform's, and the paper's displaced-jets picture is reproduced end to end.
"""

import collections
import math

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

VG = collections.namedtuple("VG", "n_x n_y x_min x_max y_min y_max")
V64 = VG(64, 64, -32.0, 32.0, -32.0, 32.0)
LINE_GRID = synth.Grid(256, 64, 1, -40.0, 40.0, -0.0005, 0.0005)


def _cell(v, x, y):
    return (int(math.floor((x - v.x_min) / ((v.x_max - v.x_min) / v.n_x))),
            int(math.floor((y - v.y_min) / ((v.y_max - v.y_min) / v.n_y))))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lines_through_a_point_meet_in_its_cell(oracle_mod, seed):
    """Candidates whose cells contain lines through a vertex V (d0 of each
    phi row's line through V, binned) all pass within half a d0 bin of V, so
    the vertex accumulator peaks at V's cell (or a neighbour) with most of
    their votes."""
    rng = np.random.default_rng(seed)
    c, s, d = oracle_mod.tables(LINE_GRID)
    dw = (LINE_GRID.d0_max - LINE_GRID.d0_min) / LINE_GRID.n_d0
    for _ in range(5):
        xv, yv = rng.uniform(-25, 25, 2)
        rows = rng.choice(LINE_GRID.n_phi, 40, replace=False)
        pk = np.array([(0, i, int((yv * c[i] - xv * s[i] - LINE_GRID.d0_min) / dw), 0, 9) for i in rows],
                      oracle_mod.PEAK_DTYPE)
        acc = oracle_mod.vertex_vote(LINE_GRID, V64, pk, 1)[0]
        a, b = np.unravel_index(np.argmax(acc), acc.shape)
        ta, tb = _cell(V64, xv, yv)
        assert abs(a - ta) <= 1 and abs(b - tb) <= 1, ((a, b), (ta, tb))
        assert acc.max() >= 0.5 * len(rows)


def test_each_vote_lies_on_its_line(oracle_mod):
    """One candidate: along the walked axis every column holds at most one
    vote, the voted cell contains the line's crossing of that column's centre
    (computed here independently), and every column whose crossing falls
    inside the grid is voted."""
    c, s, d = oracle_mod.tables(LINE_GRID)
    wx = (V64.x_max - V64.x_min) / V64.n_x
    wy = (V64.y_max - V64.y_min) / V64.n_y
    for i, j in ((3, 20), (64, 31), (100, 5), (190, 50), (250, 40)):
        pk = np.array([(0, i, j, 0, 9)], oracle_mod.PEAK_DTYPE)
        acc = oracle_mod.vertex_vote(LINE_GRID, V64, pk, 1)[0]
        cc, ss, dd = float(c[i]), float(s[i]), float(d[j])
        if abs(cc) >= abs(ss):
            for a in range(V64.n_x):
                X = V64.x_min + (a + 0.5) * wx
                Y = (dd + X * ss) / cc
                b = math.floor((Y - V64.y_min) / wy)
                col = acc[a]
                assert col.sum() == (1 if 0 <= b < V64.n_y else 0)
                if 0 <= b < V64.n_y:
                    assert col[b] == 1
        else:
            for b in range(V64.n_y):
                Y = V64.y_min + (b + 0.5) * wy
                X = (Y * cc - dd) / ss
                a = math.floor((X - V64.x_min) / wx)
                row = acc[:, b]
                assert row.sum() == (1 if 0 <= a < V64.n_x else 0)
                if 0 <= a < V64.n_x:
                    assert row[a] == 1


def test_vertex_peak_rule(oracle_mod):
    v = VG(5, 6, 0.0, 5.0, 0.0, 6.0)
    acc = np.zeros((2, 5, 6), np.uint32)
    acc[0, 2, 3] = 7
    acc[0, 2, 4] = 7          # plateau: only the lower linear index wins
    acc[0, 0, 0] = 9          # corner, no wrap to (4, 5)
    acc[0, 4, 5] = 9
    acc[1, 1, 1] = 4          # below threshold 5
    acc[1, 3, 3] = 5
    acc[1, 0, 0] = 6          # x does not wrap: (0, 0) and (4, 0) are not neighbours
    acc[1, 4, 0] = 8
    vp = oracle_mod.vertex_peaks(v, acc, 5)
    got = [tuple(int(t) for t in r) for r in vp]
    assert got == [(0, 0, 0, 9), (0, 2, 3, 7), (0, 4, 5, 9), (1, 0, 0, 6), (1, 3, 3, 5), (1, 4, 0, 8)]


def test_displaced_jets_find_their_vertices(oracle_mod):
    """The paper's demonstration: four jets of high-momentum tracks, each
    from its own displaced vertex.  The first transform finds the tracks;
    voting their candidates into the (x, y) grid puts a vertex peak within
    two cells of every true vertex, which holds the most votes around it."""
    rng = np.random.default_rng(11)
    verts = [(12.0, 5.0), (-9.0, 14.0), (-15.0, -11.0), (6.0, -18.0)]
    phi0, d0, kap = [], [], []
    for xv, yv in verts:
        axis = math.atan2(yv, xv)
        for _ in range(8):
            psi = axis + rng.uniform(-0.6, 0.6)
            phi0.append(psi % (2 * math.pi))
            d0.append(yv * math.cos(psi) - xv * math.sin(psi))
            kap.append(rng.uniform(-1e-5, 1e-5))
    x, y, _, ok = synth.helix_hits(phi0, d0, kap, synth.LAYERS_13)
    hx, hy = x[ok].astype(np.float32), y[ok].astype(np.float32)
    acc = oracle_mod.vote(LINE_GRID, hx, hy)
    pk = oracle_mod.peaks(LINE_GRID, acc, 9)
    assert len(pk) >= 32
    vacc = oracle_mod.vertex_vote(LINE_GRID, V64, pk, 1)
    vp = oracle_mod.vertex_peaks(V64, vacc, 4)
    for xv, yv in verts:
        ta, tb = _cell(V64, xv, yv)
        near = vp[(np.abs(vp["i_x"] - ta) <= 2) & (np.abs(vp["i_y"] - tb) <= 2)]
        assert len(near) > 0, (xv, yv)
        assert near["votes"].max() >= 8
