"""Seeded synthetic trigger events for the Hough-transform track finder.

This module is the shared *input* fixture: it turns seeded random track
parameters into detector hits and nothing else.  It holds none of the Hough
transform's arithmetic (no voting, no binning, no peak finding), so the CPU
oracle and the CUDA path can both be fed from it without sharing any of the
method's code.  It imports only numpy.

Detector and track model (transverse plane, the setting of the paper's toy
simulation in Section 3, extended to the displaced, curved 3-parameter helix
that Section 3 names as the next step):

* barrel layers are circles of radius ``r`` around the beam line;
* a track with perigee parameters (phi0, d0, kappa) passes its point of closest
  approach P = d0 * n, n = (-sin phi0, cos phi0), moving along
  t = (cos phi0, sin phi0), and turns toward +n when kappa > 0; its centre is
  (d0 + 1/kappa) * n and its radius 1/|kappa|;
* kappa [1/cm] = 0.0114 * Q / pT [GeV] (3.8 T field), Q = +-1;
* the hit on a layer of radius r lies on the outgoing half-turn at the arc
  length s with 1 - cos(kappa s) = (r^2 - d0^2) kappa^2 / (2 (1 + kappa d0)),
  z = z0 + s sinh(eta);
* each hit is smeared along its layer circle by N(0, sigma_rphi)/r radians;
* noise hits sit on a uniformly chosen layer at phi ~ U[0, 2 pi),
  z ~ U[-300, 300] cm.

Everything is computed in float64 and rounded to float32 once.  Hits of one
event are shuffled with the event's generator so that no ordering is implied.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

LAYERS_10 = (4.4, 7.3, 10.2, 25.5, 33.9, 41.8, 49.8, 60.8, 69.2, 78.0)
LAYERS_13 = LAYERS_10 + (86.8, 96.5, 108.0)

KAPPA_PER_INV_GEV = 0.0114  # kappa [1/cm] = 0.0114 * Q / pT at 3.8 T


@dataclasses.dataclass(frozen=True)
class Grid:
    """Accumulator binning: n_phi x n_d0 x n_kappa cells, kappa fastest."""

    n_phi: int
    n_d0: int
    n_kappa: int
    d0_min: float
    d0_max: float
    kappa_min: float
    kappa_max: float

    @property
    def n_cells(self) -> int:
        return self.n_phi * self.n_d0 * self.n_kappa


@dataclasses.dataclass(frozen=True)
class EventSpec:
    """Generator recipe for one workload's events."""

    layers: tuple
    n_tracks: str              # "fixed:N", "split:Nprompt:Ndisplaced" or "lognormal:median:sigma:lo:hi"
    displaced_frac: float      # probability a track is displaced (ignored for "split")
    d0_prompt: tuple           # ("normal", sigma) or ("uniform", lo, hi)
    d0_displaced: tuple        # ("uniform", lo, hi)
    pt: tuple                  # ("uniform", lo, hi) or ("inv2", lo, hi): density ~ 1/pT^2
    noise: str                 # "fixed:N" or "frac:F" (noise fraction of all hits)
    sigma_rphi: float = 0.01   # cm
    z0_sigma: float = 5.0      # cm
    eta_max: float = 2.5


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    grid: Grid
    spec: EventSpec
    n_events: int
    seed: int
    threshold: int
    window: int = 1


# The five workloads.  Sizes, distributions and seeds follow the batch, serving
# and stress configurations the library is measured on; values the recipe
# leaves open are the readings recorded with the design notes (d0/kappa ranges
# of the batch grids, 1/pT^2 spectra, lognormal sigma = 1, threshold 9 and
# association window 1 where unstated).
WORKLOADS = {
    "single_event_10trk": Workload(
        name="single_event_10trk",
        grid=Grid(64, 8, 64, -10.0, 10.0, -0.0114, 0.0114),
        spec=EventSpec(LAYERS_10, "fixed:10", 0.0, ("uniform", -2.0, 2.0),
                       ("uniform", -2.0, 2.0), ("uniform", 1.0, 20.0), "fixed:50"),
        n_events=1, seed=0, threshold=8),
    "dense_event_500trk": Workload(
        name="dense_event_500trk",
        grid=Grid(512, 64, 256, -25.0, 25.0, -0.0114, 0.0114),
        spec=EventSpec(LAYERS_13, "split:480:20", 0.0, ("normal", 0.01),
                       ("uniform", -20.0, 20.0), ("inv2", 1.0, 100.0), "fixed:2000"),
        n_events=1, seed=1, threshold=9),
    "batch_4096_lognormal": Workload(
        name="batch_4096_lognormal",
        grid=Grid(256, 32, 128, -25.0, 25.0, -0.0114, 0.0114),
        spec=EventSpec(LAYERS_13, "lognormal:150:1.0:20:2000", 0.05, ("normal", 0.01),
                       ("uniform", -20.0, 20.0), ("inv2", 1.0, 100.0), "frac:0.2"),
        n_events=4096, seed=2, threshold=9),
    "pileup_64x5000trk": Workload(
        name="pileup_64x5000trk",
        grid=Grid(1024, 128, 512, -35.0, 35.0, -0.01425, 0.01425),
        spec=EventSpec(LAYERS_13, "fixed:5000", 0.30, ("normal", 0.01),
                       ("uniform", -30.0, 30.0), ("inv2", 0.8, 100.0), "fixed:15000"),
        n_events=64, seed=3, threshold=10),
    "serving_lognormal": Workload(
        name="serving_lognormal",
        grid=Grid(256, 32, 128, -25.0, 25.0, -0.0114, 0.0114),
        spec=EventSpec(LAYERS_13, "lognormal:150:1.0:20:2000", 0.05, ("normal", 0.01),
                       ("uniform", -20.0, 20.0), ("inv2", 1.0, 100.0), "frac:0.2"),
        n_events=4096, seed=4, threshold=9),
}


@dataclasses.dataclass
class Batch:
    """Ragged-packed SoA hits of several events (the library's input layout)."""

    x: np.ndarray            # float32 [n_hits]
    y: np.ndarray            # float32 [n_hits]
    z: np.ndarray            # float32 [n_hits]
    layer: np.ndarray        # int8    [n_hits]
    event_offsets: np.ndarray  # int32 [n_events + 1]
    layer_r: np.ndarray      # float32 [n_layers]
    truth_track: Optional[np.ndarray] = None  # int32 [n_hits], -1 for noise, else track index within event
    truth_params: Optional[list] = None       # per event: float64 [n_tracks, 3] (phi0, d0, kappa)

    @property
    def n_events(self) -> int:
        return int(self.event_offsets.shape[0] - 1)

    @property
    def n_hits(self) -> int:
        return int(self.x.shape[0])

    def event(self, e: int) -> "Batch":
        lo, hi = int(self.event_offsets[e]), int(self.event_offsets[e + 1])
        return Batch(self.x[lo:hi].copy(), self.y[lo:hi].copy(), self.z[lo:hi].copy(),
                     self.layer[lo:hi].copy(), np.array([0, hi - lo], dtype=np.int32),
                     self.layer_r,
                     None if self.truth_track is None else self.truth_track[lo:hi].copy(),
                     None if self.truth_params is None else [self.truth_params[e]])

    def select(self, events) -> "Batch":
        return concat([self.event(int(e)) for e in events])


def concat(batches) -> Batch:
    """Pack several batches into one (event order preserved).  The layer
    radii of the result are the longest of the batches' tables; every other
    table must be a prefix of it, so that each hit's layer id stays valid."""
    batches = list(batches)
    if not batches:
        raise ValueError("concat needs at least one batch")
    layer_r = max((np.asarray(b.layer_r, np.float32) for b in batches), key=len)
    for b in batches:
        lr = np.asarray(b.layer_r, np.float32)
        if not np.array_equal(lr, layer_r[:len(lr)]):
            raise ValueError("concat: layer radii differ between batches")
    offs = [0]
    for b in batches:
        base = offs[-1]
        offs.extend(int(base + o) for o in b.event_offsets[1:])
    tt = None
    if all(b.truth_track is not None for b in batches):
        tt = np.concatenate([b.truth_track for b in batches]).astype(np.int32)
    tp = None
    if all(b.truth_params is not None for b in batches):
        tp = [p for b in batches for p in b.truth_params]
    return Batch(np.concatenate([b.x for b in batches]).astype(np.float32),
                 np.concatenate([b.y for b in batches]).astype(np.float32),
                 np.concatenate([b.z for b in batches]).astype(np.float32),
                 np.concatenate([b.layer for b in batches]).astype(np.int8),
                 np.asarray(offs, dtype=np.int32), layer_r, tt, tp)


def _draw_pt(rng, spec, n):
    kind, lo, hi = spec.pt
    u = rng.random(n)
    if kind == "uniform":
        return lo + (hi - lo) * u
    if kind == "inv2":  # density ~ 1/pT^2 on [lo, hi]: inverse CDF
        return 1.0 / (1.0 / lo - u * (1.0 / lo - 1.0 / hi))
    raise ValueError(kind)


def _draw_d0(rng, dist, n):
    if n == 0:
        return np.zeros(0)
    if dist[0] == "normal":
        return rng.normal(0.0, dist[1], n)
    if dist[0] == "uniform":
        return rng.uniform(dist[1], dist[2], n)
    raise ValueError(dist[0])


def _n_tracks(rng, spec):
    kind, *args = spec.n_tracks.split(":")
    if kind == "fixed":
        return int(args[0]), None
    if kind == "split":
        return int(args[0]) + int(args[1]), int(args[1])
    if kind == "lognormal":
        med, sig, lo, hi = float(args[0]), float(args[1]), int(args[2]), int(args[3])
        return int(np.clip(np.rint(med * math.exp(rng.normal(0.0, sig))), lo, hi)), None
    raise ValueError(kind)


def helix_hits(phi0, d0, kappa, layers):
    """Exact (float64) transverse crossing points of perigee helices with layers.

    Returns (x, y, s, ok), each [n_tracks, n_layers]; ``ok`` marks layers the
    outgoing half-turn reaches (|d0| < r <= |d0 + 2/kappa|).
    """
    phi0 = np.asarray(phi0, dtype=np.float64)[:, None]
    d0 = np.asarray(d0, dtype=np.float64)[:, None]
    kappa = np.asarray(kappa, dtype=np.float64)[:, None]
    r = np.asarray(layers, dtype=np.float64)[None, :]
    one_m_cos = (r * r - d0 * d0) * kappa * kappa / (2.0 * (1.0 + kappa * d0))
    ok = (r > np.abs(d0)) & (one_m_cos >= 0.0) & (one_m_cos <= 2.0) & (1.0 + kappa * d0 > 0.0)
    theta = np.arccos(np.clip(1.0 - one_m_cos, -1.0, 1.0))         # |kappa| s in [0, pi]
    s = theta / np.abs(kappa)
    along = np.sin(theta) / np.abs(kappa)                           # component along t
    across = d0 + one_m_cos / kappa                                 # component along n
    c, sn = np.cos(phi0), np.sin(phi0)
    x = along * c - across * sn
    y = along * sn + across * c
    return x, y, s, ok


def generate_event(rng: np.random.Generator, spec: EventSpec):
    """One event: (x, y, z, layer, truth_track, params[n_tracks, 3])."""
    nt, n_disp = _n_tracks(rng, spec)
    if n_disp is None:
        displaced = rng.random(nt) < spec.displaced_frac
    else:
        displaced = np.zeros(nt, dtype=bool)
        displaced[nt - n_disp:] = True
    pt = _draw_pt(rng, spec, nt)
    q = np.where(rng.random(nt) < 0.5, -1.0, 1.0)
    kappa = KAPPA_PER_INV_GEV * q / pt
    phi0 = rng.uniform(0.0, 2.0 * math.pi, nt)
    d0 = np.where(displaced, _draw_d0(rng, spec.d0_displaced, nt), _draw_d0(rng, spec.d0_prompt, nt))
    z0 = rng.normal(0.0, spec.z0_sigma, nt)
    eta = rng.uniform(-spec.eta_max, spec.eta_max, nt)
    layers = np.asarray(spec.layers, dtype=np.float64)
    hx, hy, hs, ok = helix_hits(phi0, d0, kappa, layers)
    # r-phi smear: rotate each hit along its own layer circle
    rr = np.broadcast_to(layers[None, :], hx.shape)
    ang = np.arctan2(hy, hx) + rng.normal(0.0, spec.sigma_rphi, hx.shape) / rr
    hx, hy = rr * np.cos(ang), rr * np.sin(ang)
    hz = z0[:, None] + hs * np.sinh(eta)[:, None]
    ti, li = np.nonzero(ok)
    x, y, z = hx[ti, li], hy[ti, li], hz[ti, li]
    lay = li.astype(np.int8)
    truth = ti.astype(np.int32)
    kind, val = spec.noise.split(":")
    if kind == "fixed":
        nn = int(val)
    else:  # noise is a fraction F of all hits: nn = F/(1-F) * track hits
        f = float(val)
        nn = int(round(x.shape[0] * f / (1.0 - f)))
    nl = rng.integers(0, layers.shape[0], nn)
    nphi = rng.uniform(0.0, 2.0 * math.pi, nn)
    x = np.concatenate([x, layers[nl] * np.cos(nphi)])
    y = np.concatenate([y, layers[nl] * np.sin(nphi)])
    z = np.concatenate([z, rng.uniform(-300.0, 300.0, nn)])
    lay = np.concatenate([lay, nl.astype(np.int8)])
    truth = np.concatenate([truth, np.full(nn, -1, dtype=np.int32)])
    perm = rng.permutation(x.shape[0])
    params = np.stack([phi0, d0, kappa], axis=1)
    return (x[perm].astype(np.float32), y[perm].astype(np.float32), z[perm].astype(np.float32),
            lay[perm], truth[perm], params)


def generate(workload: Workload, n_events: Optional[int] = None, seed: Optional[int] = None,
             first_event: int = 0) -> Batch:
    """Events ``first_event .. first_event + n_events - 1`` of a workload.

    Event e draws from ``default_rng([seed, e])`` so any subset of a workload
    can be regenerated on its own (the parity tests sample events this way).
    """
    n = workload.n_events if n_events is None else int(n_events)
    sd = workload.seed if seed is None else int(seed)
    xs, ys, zs, ls, ts, ps, offs = [], [], [], [], [], [], [0]
    for e in range(first_event, first_event + n):
        rng = np.random.default_rng([sd, e])
        x, y, z, lay, truth, params = generate_event(rng, workload.spec)
        xs.append(x); ys.append(y); zs.append(z); ls.append(lay); ts.append(truth); ps.append(params)
        offs.append(offs[-1] + x.shape[0])
    cat = (lambda a, dt: np.concatenate(a).astype(dt)) if n else (lambda a, dt: np.zeros(0, dt))
    return Batch(cat(xs, np.float32), cat(ys, np.float32), cat(zs, np.float32), cat(ls, np.int8),
                 np.asarray(offs, dtype=np.int32), np.asarray(workload.spec.layers, dtype=np.float32),
                 cat(ts, np.int32), ps)


def from_arrays(x, y, layer=None, z=None, event_offsets=None, layer_r=LAYERS_13) -> Batch:
    """Wrap hand-made hit arrays (tests, examples) as a Batch."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    n = x.shape[0]
    z = np.zeros(n, np.float32) if z is None else np.ascontiguousarray(z, dtype=np.float32)
    layer = np.zeros(n, np.int8) if layer is None else np.ascontiguousarray(layer, dtype=np.int8)
    offs = np.array([0, n], np.int32) if event_offsets is None else np.asarray(event_offsets, np.int32)
    return Batch(x, y, z, layer, offs, np.asarray(layer_r, dtype=np.float32))
