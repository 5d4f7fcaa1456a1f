#!/usr/bin/env python3
"""Benchmark: events/s of the whole Hough-transform path on one GB300.

One step = vote + peaks + association of one batch of 4096 ragged synthetic
trigger events (tracks/event lognormal, median 150; 256 x 32 x 128 grid;
threshold 9, window 1), run as one persistent launch per kernel and wave,
replayed from a CUDA graph.  Inputs are resident in HBM when the timed region
starts; the L2 is flushed between timed steps.  Also reported: the plain
one-event-per-launch form on a sample of the same batch, the end-to-end rate
through the C ABI with pinned host buffers (copies inside the timed region),
the dense single event and the pileup batch, the dominant kernels against
their rooflines, the flip fraction of a plain float32 evaluation, and the CPU
oracle on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Under torchrun each rank processes its own batch (weak scaling, no collective).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batch_4096_lognormal"
METRIC = "events/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) per hit of one launch on the first 64 events of
# the batch workload (275,323 hits), from one ncu capture of the kernels as
# they are now (vote_band_kernel<4, 128, 1, 0> writing records: 0.164465 GB
# read + 1.322960 GB written; assoc_rec_kernel<4, 2>: 1.766159 + 0.443076 GB);
# set to None when a kernel changes until it is captured again
PROFILE_HITS = 275323
VOTE_DRAM_PER_HIT = (0.081700 + 1.241773) * 1e9 / PROFILE_HITS
ASSOC_DRAM_PER_HIT = (1.766159 + 0.443076) * 1e9 / PROFILE_HITS
# FP32 lane operations per (hit, phi0, d0) cell of the method: 8 arithmetic
# (q: 2 products and a difference; a = q - d; den: d^2 and 2dq terms, 3; the
# kappa scale) + 1 IEEE division + 4 compare/convert (den > 0, w >= 0,
# w < n_kappa, the floor)
OPS_PER_CELL = 13


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(w, rank):
    """Generator seed of a rank's batch: rank 0 the workload's own, every
    other rank its own stream (weak scaling: the same shape, other events)."""
    return w.seed + 1000 * rank if rank else None


def max_over_ranks(x, world, device):
    """The largest value of a time-like float over the ranks (identity at
    one rank); `device` is where the process group's backend reduces."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_single_thread():
    """The oracle on one host thread, on the whole single event, the whole
    dense event and a 4-event subset of the batch (extrapolated per event),
    plus the flip fraction of the plain float32 evaluation against the
    binary64 bins on a sample of every workload.  Run after every GPU
    measurement: host work beside the timed end-to-end pass disturbed it."""
    import oracle
    from paper_1311_2769_gb300 import synth
    oracle.build()
    out = {"threads": 1, "events": {}, "flip_fraction_plain_fp32": {}}
    for name, n in (("single_event_10trk", 1), ("batch_4096_lognormal", 4), ("dense_event_500trk", 1)):
        w = synth.WORKLOADS[name]
        b = synth.generate(w, n_events=n)
        t0 = time.perf_counter()
        votes, peaks, pairs = oracle.run_events(w.grid, b.x, b.y, b.event_offsets, w.threshold, w.window, 1)
        dt = time.perf_counter() - t0
        row = {"events": n, "hits": int(b.n_hits), "seconds": dt, "events_per_s": n / dt,
               "hit_votes_per_s": float(b.n_hits) * w.grid.n_phi * w.grid.n_d0 / dt,
               "votes": votes, "peaks": peaks, "pairs": pairs}
        if n > 1:
            row["note"] = f"events 0..{n - 1} of the 4096-event batch; per-event rate extrapolated to the batch"
        out["events"][name] = row
    # plain float32 op order (no contraction) against the binary64 bins
    for name, n_hits in (("single_event_10trk", None), ("dense_event_500trk", 300), ("batch_4096_lognormal", None),
                         ("pileup_64x5000trk", 300)):
        w = synth.WORKLOADS[name]
        b = synth.generate(w, n_events=1)
        x, y = b.x, b.y
        if n_hits and len(x) > n_hits:
            sel = np.random.default_rng(1).choice(len(x), n_hits, replace=False)
            x, y = x[sel], y[sel]
        v64, v32, diff = oracle.flip_count(w.grid, x, y)
        out["flip_fraction_plain_fp32"][name] = {"binary64_votes": v64, "columns_differing": diff,
                                                 "fraction": diff / max(v64, 1), "hits": int(len(x)),
                                                 "sample": "event 0" + (f", {n_hits} random hits" if n_hits else "")}
    return out


def cpu_baseline(w, batch, budget_s=15.0):
    """The oracle as it stands, event-parallel on every host core (largest
    event first, one event at a time per thread), on a prefix of the
    workload's events whose length is a multiple of the core count and at
    least four events per core (sized to about budget_s seconds)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    # calibrate on one event per core, then size the sample
    n = min(cores, batch.n_events)
    sub = batch.select(range(n))
    t0 = time.perf_counter()
    oracle.run_events(w.grid, sub.x, sub.y, sub.event_offsets, w.threshold, w.window, cores)
    dt = time.perf_counter() - t0
    per_event = dt * cores / n
    want = int(budget_s * cores / max(per_event, 1e-9))
    want = max(4 * cores, (want // cores) * cores)
    want = min(want, batch.n_events)
    sub = batch.select(range(want))
    t0 = time.perf_counter()
    votes, peaks, pairs = oracle.run_events(w.grid, sub.x, sub.y, sub.event_offsets, w.threshold, w.window, cores)
    dt = time.perf_counter() - t0
    out = {"value": want / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": f"events 0..{want - 1} of the 4096-event batch ({sub.n_hits} hits), "
                     f"vote+peaks+association, one event per thread, largest first", "seconds": dt,
           "hit_votes_per_s": float(sub.n_hits) * w.grid.n_phi * w.grid.n_d0 / dt,
           "all_cores": {"threads": cores, "events": want, "events_per_s": want / dt}}
    return out


def vote_ceilings(ht, g, batch, w, cells, vote_s, vote_traffic, peaks, dev, sample_events=64):
    """The vote kernel against each ceiling it could meet, every ceiling
    measured here: FP32 issue (OPS_PER_CELL lane operations per cell), IEEE
    division (one per cell), shared-memory increments (one per accepted vote;
    the accepted fraction of cells is counted on the first `sample_events`
    events) and HBM (its ncu DRAM traffic).  `binding` names the largest
    fraction."""
    rates = {"fp32_ops_per_s": ht.ht_microbench(ht.HT_MB_FP32, 160000),
             "shared_red_per_s": ht.ht_microbench(ht.HT_MB_SHARED_RED, 40000),
             "fdiv_per_s": ht.ht_microbench(ht.HT_MB_FDIV, 40000)}
    sub = batch.select(range(min(sample_events, batch.n_events)))
    c2 = ht.Context(g, w.spec.layers)
    c2.vote(ht.Hits.from_batch(sub, device=dev))
    votes = sum(int(c2.accumulator(e).sum(dtype=np.int64)) for e in range(sub.n_events))
    c2.close()
    accepted = votes / (float(sub.n_hits) * g.n_phi * g.n_d0)
    frac = {"issue": float(OPS_PER_CELL) * cells / vote_s / rates["fp32_ops_per_s"],
            "shared_atomic": accepted * cells / vote_s / rates["shared_red_per_s"]}
    if vote_traffic and peaks.get("hbm_gbs"):
        frac["hbm"] = vote_traffic / vote_s / (peaks["hbm_gbs"] * 1e9)
    # the method divides once per cell; the kernel replaces the IEEE division
    # by a certified reciprocal estimate, so this ratio is not a bound on it
    divide = cells / vote_s / rates["fdiv_per_s"]
    return {"kernel": "vote_band_kernel", "frac": frac, "binding": max(frac, key=frac.get),
            "cells_over_ieee_divide_rate": divide, "accepted_votes_per_cell": accepted,
            "sample": f"events 0..{sub.n_events - 1}", "measured": rates}


def track_efficiency(g, batch, pk, min_hits=8):
    """(found, findable): tracks with >= min_hits hits whose true (phi0, d0,
    kappa) lies inside the grid, found when a peak of their event lies within
    one cell of the true cell in every axis (phi0 periodic)."""
    dphi = 2 * math.pi / g.n_phi
    dd = (g.d0_max - g.d0_min) / g.n_d0
    dk = (g.kappa_max - g.kappa_min) / g.n_kappa
    ev = pk["event"]
    found = findable = 0
    for e in range(batch.n_events):
        lo, hi = batch.event_offsets[e], batch.event_offsets[e + 1]
        nh = np.bincount(batch.truth_track[lo:hi][batch.truth_track[lo:hi] >= 0],
                         minlength=len(batch.truth_params[e]))
        P = batch.truth_params[e]
        ok = (nh >= min_hits) & (P[:, 1] >= g.d0_min) & (P[:, 1] < g.d0_max) & (P[:, 2] >= g.kappa_min) & (
            P[:, 2] < g.kappa_max)
        if not ok.any():
            continue
        i = ((P[ok, 0] % (2 * math.pi)) / dphi).astype(np.int64)
        j = ((P[ok, 1] - g.d0_min) / dd).astype(np.int64)
        k = ((P[ok, 2] - g.kappa_min) / dk).astype(np.int64)
        findable += int(ok.sum())
        sel = pk[ev == e]
        if len(sel) == 0:
            continue
        di = np.abs(sel["i_phi"][None, :].astype(np.int64) - i[:, None])
        di = np.minimum(di, g.n_phi - di)
        near = (di <= 1) & (np.abs(sel["i_d0"][None, :] - j[:, None]) <= 1) & (
            np.abs(sel["i_kappa"][None, :] - k[:, None]) <= 1)
        found += int(near.any(axis=1).sum())
    return found, findable


def range_vote_report(dev, n_batch=256, n_single=64):
    """Point against range voting: device step time and track-finding
    efficiency on a sample of the batch workload and of the single-event
    workload (coarse 64-row grid), at each workload's threshold."""
    from paper_1311_2769_gb300 import ht, synth
    out = {}
    for wname, n in (("batch_4096_lognormal", n_batch), ("single_event_10trk", n_single)):
        w = synth.WORKLOADS[wname]
        b = synth.generate(w, n_events=n)
        hits = ht.Hits.from_batch(b, device=dev)
        rows = {}
        for mode, name in ((ht.HT_VOTE_POINT, "point"), (ht.HT_VOTE_RANGE, "range")):
            ctx = ht.Context(w.grid, w.spec.layers)
            ctx.set_option(ht.HT_OPT_VOTE_MODE, mode)
            ctx.set_option(ht.HT_OPT_PHASE_TIMING, 1)
            res = ht.Results(n * 200000 + 4096, n * 6000000 + 65536, device=dev)
            ts = []
            for it in range(4):
                ctx.process(hits, w.threshold, w.window, res)
                ctx.sync()
                if it:
                    ts.append(ctx.phase_times())
            pk, _, hidx = res.host()
            f, fa = track_efficiency(w.grid, b, pk)
            rows[name] = {"ms_per_event": float(np.mean([t[2] for t in ts])) / n,
                          "vote_ms": float(np.mean([t[0] for t in ts])),
                          "peaks_assoc_ms": float(np.mean([t[1] for t in ts])),
                          "peaks_per_event": len(pk) / n, "pairs_per_event": len(hidx) / n,
                          "tracks_found": f, "tracks_findable": fa, "efficiency": f / max(fa, 1)}
            ctx.close()
        out[wname] = {"events": n, "threshold": w.threshold, **rows}
    return out


def vertex_report(dev, n_jets=64, n_batch=512):
    """Second Hough transform: device time and vertex finding on events of
    four displaced jets of straight tracks (the paper's picture; a true
    vertex counts as found when a vertex lies within two cells), and device
    time on a sample of the batch workload's candidates."""
    import collections
    import torch
    from paper_1311_2769_gb300 import ht, synth
    VG = collections.namedtuple("VG", "n_x n_y x_min x_max y_min y_max")
    vg = VG(64, 64, -32.0, 32.0, -32.0, 32.0)
    rng = np.random.default_rng(2024)
    xs, ys, offs, verts = [], [], [0], []
    for _ in range(n_jets):
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
    jets = synth.from_arrays(np.concatenate(xs), np.concatenate(ys), event_offsets=np.array(offs, np.int32))
    out = {}
    for name, b, g, thr, vthr in (
            ("displaced_jets", jets, synth.Grid(256, 64, 1, -40.0, 40.0, -0.0005, 0.0005), 9, 6),
            ("batch_4096_lognormal", synth.generate(synth.WORKLOADS[WORKLOAD], n_events=n_batch),
             synth.WORKLOADS[WORKLOAD].grid, synth.WORKLOADS[WORKLOAD].threshold, 40)):
        ctx = ht.Context(g, synth.LAYERS_13)
        if name == "displaced_jets":  # straight tracks: the paper's kappa = 0 model
            ctx.set_option(ht.HT_OPT_VOTE_MODE, ht.HT_VOTE_LINE)
            ctx.set_option(ht.HT_OPT_PHASE_TIMING, 1)
        res = ht.Results(b.n_events * 20000 + 4096, b.n_events * 800000 + 65536, device=dev)
        for _ in range(2):
            ctx.process(ht.Hits.from_batch(b, device=dev), thr, 1, res)
            ctx.sync()
        step = ctx.phase_times()[2] if name == "displaced_jets" else None
        ms = []
        s = torch.cuda.current_stream()
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            vo, cnt = ctx.vertices(vg, res, vthr, cap=1 << 20, stream=s)
            e1.record(s)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        n = int(cnt.item())
        row = {"events": b.n_events, "candidates": int(res.counts[0].item()), "vertex_threshold": vthr,
               "ms": float(np.median(ms)), "vertices": n}
        if step is not None:
            row["line_vote_step_ms"] = step
        if name == "displaced_jets":
            got = ht.vertices_host(vo, min(n, 1 << 20))
            found = 0
            for e, vs in enumerate(verts):
                ev = got[got["event"] == e]
                for xv, yv in vs:
                    a, c = int((xv + 32.0) // 1.0), int((yv + 32.0) // 1.0)
                    found += int(np.any((np.abs(ev["i_x"] - a) <= 2) & (np.abs(ev["i_y"] - c) <= 2)))
            row["true_vertices"] = 4 * len(verts)
            row["found"] = found
        out[name] = row
        ctx.close()
    return out


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores (rank 0 only)."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_1311_2769_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n_sample = 4 * cores  # four events per core, handed out largest first
    batch = synth.generate(w, n_events=n_sample)
    for _ in range(args.warmup):
        sub = batch.select(range(min(cores, n_sample)))
        oracle.run_events(w.grid, sub.x, sub.y, sub.event_offsets, w.threshold, w.window, cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run_events(w.grid, batch.x, batch.y, batch.event_offsets, w.threshold, w.window, cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.median(times))
    value = n_sample / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_step": n_sample, "grid": [256, 32, 128],
                       "threshold": w.threshold, "window": w.window},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": METRIC,
                             "sample": f"events 0..{n_sample - 1} of the 4096-event batch per step, "
                                       f"one event at a time per thread, largest first"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _median_ms(fn, stream, flush, reps):
    """Median device time (CUDA events on `stream`) of `fn` over reps calls,
    the L2 flushed before each."""
    import torch
    ms = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms)), ms


def secondary_workloads(dev, stream, flush, reps=5):
    """The single 10-track event (150 hits, 64 x 8 x 64 grid), the dense
    single event (8.5k hits, 512 x 64 x 256 grid) and the pileup batch (64
    events of ~76k hits, 1024 x 128 x 512 grid, accumulators admitted four
    events at a time), each timed as whole steps on the device (median of
    `reps`, 21 for the small event, 3 for pileup, L2 flushed before each)."""
    from paper_1311_2769_gb300 import ht, synth
    out = {}
    for name, waves_of, r in (("single_event_10trk", 0, 21), ("dense_event_500trk", 0, reps),
                              ("pileup_64x5000trk", 4, 3)):
        w = synth.WORKLOADS[name]
        g = w.grid
        b = synth.generate(w)
        ctx = ht.Context(g, w.spec.layers)
        if waves_of:
            ctx.set_option(ht.HT_OPT_ACC_BUDGET, waves_of * 4 * g.n_phi * g.n_d0 * g.n_kappa)
        hits = ht.Hits.from_batch(b, device=dev)
        probe = ht.Results(1 << 20, 1 << 20, device=dev)
        ctx.process(hits, w.threshold, w.window, probe, stream)
        ctx.sync(allow_overflow=True)
        n_peaks, n_pairs = (int(v) for v in probe.counts.cpu().numpy())
        del probe
        res = ht.Results(n_peaks + 1024, n_pairs + 4096, device=dev)
        step = lambda: ctx.process(hits, w.threshold, w.window, res, stream)
        step()
        ctx.sync()
        med, all_ms = _median_ms(step, stream, flush, r)
        out[name] = {"events": b.n_events, "hits": int(b.n_hits), "grid": [g.n_phi, g.n_d0, g.n_kappa],
                     "threshold": w.threshold, "ms_per_step": med, "events_per_s": b.n_events / (med / 1e3),
                     "hit_votes_per_s": float(b.n_hits) * g.n_phi * g.n_d0 / (med / 1e3),
                     "peaks": n_peaks, "pairs": n_pairs, "waves": ctx.get_option(ht.HT_OPT_WAVES),
                     "records": ctx.get_option(ht.HT_OPT_RECORDS), "runs_ms": all_ms}
        ctx.close()
        del res, hits
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()

    from paper_1311_2769_gb300 import build, ht, synth

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    w = synth.WORKLOADS[args.workload]
    g = w.grid
    batch = synth.generate(w, n_events=args.events, seed=rank_seed(w, rank))
    n_events, n_hits = batch.n_events, batch.n_hits
    cols = g.n_phi * g.n_d0
    hit_votes = float(n_hits) * cols

    ctx = ht.Context(g, w.spec.layers)
    ctx.set_option(ht.HT_OPT_PHASE_TIMING, 1)
    if args.waves_of:
        # accumulator memory admitted for this many events at a time (waves)
        ctx.set_option(ht.HT_OPT_ACC_BUDGET, args.waves_of * 4 * g.n_phi * g.n_d0 * g.n_kappa)
    if args.record_budget_gb:
        ctx.set_option(ht.HT_OPT_RECORD_BUDGET, int(args.record_budget_gb * 2 ** 30))
    hits_d = ht.Hits.from_batch(batch, device=dev)
    if args.prune is not None:
        ctx.set_option(ht.HT_OPT_PRUNE, args.prune)
    if args.hit_staging is not None:
        ctx.set_option(ht.HT_OPT_HIT_STAGING, args.hit_staging)
    if args.vote_items is not None:
        ctx.set_option(ht.HT_OPT_VOTE_ITEMS, args.vote_items)
    if args.band_split is not None:
        ctx.set_option(ht.HT_OPT_BAND_SPLIT, args.band_split)
    if args.tile:
        for k, v in zip((ht.HT_OPT_TILE_PHI, ht.HT_OPT_TILE_D0, ht.HT_OPT_THREADS), args.tile.split(",")):
            ctx.set_option(k, int(v))
    else:
        # autotune the tile on the batch itself (outside the timed region):
        # timings on a smaller sample ranked the tiles differently from the
        # full step
        per_ev = 4 * g.n_phi * g.n_d0 * g.n_kappa
        n_s = max(1, min(n_events, ctx.get_option(ht.HT_OPT_ACC_BUDGET) // per_ev))
        if n_s == n_events:
            ctx.autotune(hits_d)
        else:
            sample = batch.select(range(0, n_events, max(1, n_events // n_s))[:n_s])
            ctx.autotune(ht.Hits.from_batch(sample, device=dev))
    tile = {"tile_phi": ctx.get_option(ht.HT_OPT_TILE_PHI), "tile_d0": ctx.get_option(ht.HT_OPT_TILE_D0),
            "threads": ctx.get_option(ht.HT_OPT_THREADS)}
    band_split = ctx.get_option(ht.HT_OPT_BAND_SPLIT)

    # size outputs from one untimed pass
    probe = ht.Results(1 << 20, 1 << 20, device=dev)
    ctx.process(hits_d, w.threshold, w.window, probe)
    try:
        ctx.sync()
    except ht.HtError as e:
        if e.status != ht.HT_ERR_OVERFLOW:
            raise
    n_peaks, n_pairs = (int(v) for v in probe.counts.cpu().numpy())
    del probe
    res = ht.Results(int(n_peaks * 1.05) + 1024, int(n_pairs * 1.05) + 4096, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        ctx.process(hits_d, w.threshold, w.window, res, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    ctx.sync()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, vote_ms, rest_ms, assoc_ms = [], [], [], []
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            ctx.sync()
            step_ms.append(e0.elapsed_time(e1))
            v, r, _, a = ctx.phase_times()
            vote_ms.append(v)
            rest_ms.append(r)
            assoc_ms.append(a)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(float(np.mean(step_ms)), world, dev)
    launches = ctx.get_option(ht.HT_OPT_LAUNCHES)
    waves = ctx.get_option(ht.HT_OPT_WAVES)
    counts = res.counts.cpu().numpy()
    # ---- end to end through the C ABI: pinned host inputs and outputs (measured
    # right after the device steps, before the reports below allocate), in a
    # context of its own with the step's tile
    e2e = None
    if not args.no_extras:  # every rank measures its own end-to-end rate
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hx, hy, ho, hl = pin(batch.x), pin(batch.y), pin(batch.event_offsets), pin(batch.layer)
        hits_h = ht.Hits.__new__(ht.Hits)
        hits_h.arrays = (hx, hy, ho, hl)
        hits_h.struct = ht.HtHits(hx.data_ptr(), hy.data_ptr(), None, hl.data_ptr(), ho.data_ptr(), n_events,
                                  ht.HT_HOST, n_hits)
        rh = ht.Results.__new__(ht.Results)
        rh.peak_cap, rh.pair_cap = res.peak_cap, res.pair_cap
        rh.peaks = torch.empty((rh.peak_cap, 5), dtype=torch.int32).pin_memory()
        rh.peak_offsets = torch.empty(rh.peak_cap + 1, dtype=torch.int64).pin_memory()
        rh.hit_idx = torch.empty(rh.pair_cap, dtype=torch.int32).pin_memory()
        rh.counts = torch.zeros(2, dtype=torch.int64).pin_memory()
        rh.struct = ht.HtResults(rh.peaks.data_ptr(), rh.peak_cap, rh.peak_offsets.data_ptr(),
                                 rh.hit_idx.data_ptr(), rh.pair_cap, rh.counts.data_ptr(), ht.HT_HOST)
        ectx = ht.Context(g, w.spec.layers)
        for k, v in ((ht.HT_OPT_TILE_PHI, tile["tile_phi"]), (ht.HT_OPT_TILE_D0, tile["tile_d0"]),
                     (ht.HT_OPT_THREADS, tile["threads"]), (ht.HT_OPT_VOTE_ITEMS, ctx.get_option(ht.HT_OPT_VOTE_ITEMS)),
                     (ht.HT_OPT_HIT_STAGING, ctx.get_option(ht.HT_OPT_HIT_STAGING)),
                     (ht.HT_OPT_BAND_SPLIT, ctx.get_option(ht.HT_OPT_BAND_SPLIT))):
            ectx.set_option(k, v)
        if args.host_chunks:
            ectx.set_option(ht.HT_OPT_HOST_CHUNKS, args.host_chunks)
        for _ in range(2):  # warm: buffers, first DMA into the pinned pages
            ectx.process(hits_h, w.threshold, w.window, rh, stream)
        et = []
        for _ in range(max(5, min(args.steps, 9))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ectx.process(hits_h, w.threshold, w.window, rh, stream)  # synchronous (host outputs)
            et.append(time.perf_counter() - t0)
        e2e_waves = ectx.get_option(ht.HT_OPT_WAVES)
        e2e_chunks = ectx.get_option(ht.HT_OPT_HOST_CHUNKS)
        e2e_copy = ectx.get_option(ht.HT_OPT_HOST_COPY)
        ectx.close()
        c = rh.counts.numpy()
        h2d = n_hits * (4 + 4 + 1) + 4 * (n_events + 1)
        d2h = 16 + int(c[0]) * 20 + (int(c[0]) + 1) * 8 + int(c[1]) * 4
        # the box's pinned device-to-host copy-engine rate (1 GiB into the
        # result buffer; the library's copy kernel does not use the engines)
        n_copy = min(1 << 28, rh.pair_cap)
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        rh.hit_idx[:n_copy].copy_(res.hit_idx[:n_copy], non_blocking=True)
        d1.record(stream)
        d1.synchronize()
        e2e_s = max_over_ranks(float(np.median(et)), world, dev)
        e2e = {"value": world * n_events / e2e_s, "unit": METRIC, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "seconds_per_step": e2e_s, "runs_s": et, "stat": "median",
               "waves": e2e_waves, "host_chunks": e2e_chunks,
               "result_copy": f"copy kernel, {e2e_copy} blocks" if e2e_copy else "copy engines",
               "d2h_gbs": 4.0 * n_copy / (d0.elapsed_time(d1) * 1e-3) / 1e9}
        del rh, hits_h

    # circle fit of the stored candidates of the last step (not in the step)
    fit_ms = []
    for _ in range(3):
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        fits = ctx.fit(res, stream=stream)
        f1.record(stream)
        f1.synchronize()
        fit_ms.append(f0.elapsed_time(f1))
    n_fit = int(min(counts[0], res.peak_cap))
    fitted = int((fits.view(torch.int32)[0::12][:n_fit] == 1).sum().item())  # status, every 48 bytes
    # binary64 work of the fit: 23 operations per row hit (14 for the sums,
    # 9 for the residual, its square root counted as one) + ~45 per candidate
    fp64_rate = ht.ht_microbench(ht.HT_MB_FP64, 2500)
    fit_ops = 23.0 * float(min(counts[1], res.pair_cap)) + 45.0 * n_fit
    fit_info = {"ms": float(np.median(fit_ms)), "candidates": n_fit, "fitted": fitted,
                "candidates_per_s": n_fit / (float(np.median(fit_ms)) / 1e3),
                "roofline": {"bound": "fp64", "achieved": fit_ops / (float(np.median(fit_ms)) / 1e3) / 1e12,
                             "peak": fp64_rate / 1e12, "unit": "T binary64 ops/s",
                             "frac": fit_ops / (float(np.median(fit_ms)) / 1e3) / fp64_rate,
                             "peak_basis": "measured binary64 multiply/add rate (ht_microbench)"}}
    # duplicate and mirror merging of those fits (radius 2; not in the step)
    merge_ms = []
    for _ in range(3):
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        state, kept = ctx.merge(res, fits, 2, stream=stream)
        m1.record(stream)
        m1.synchronize()
        merge_ms.append(m0.elapsed_time(m1))
    st = torch.bincount((state[:n_fit] + 2).to(torch.int64), minlength=4).cpu().numpy()
    merge_info = {"ms": float(np.median(merge_ms)), "radius": 2, "kept": int(kept.item()),
                  "duplicate": int(st[2]), "backward": int(st[1]), "unfitted": int(st[0]),
                  "candidates_per_s": n_fit / (float(np.median(merge_ms)) / 1e3)}
    del fits, state
    records = ctx.get_option(ht.HT_OPT_RECORDS)
    prune = ctx.get_option(ht.HT_OPT_PRUNE)
    # the step's context holds the batch's records and accumulators: free it
    # before the reports below allocate their own
    ctx.close()
    del res, hits_d
    torch.cuda.empty_cache()
    if args.no_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": world * n_events / (ms / 1e3), "ms_per_step": ms,
                              "workload": args.workload, "hit_votes_per_s": world * hit_votes / (ms / 1e3),
                              "prune": prune, "waves": waves, "records": records,
                              "events": n_events, "phase_ms": {"vote": float(np.mean(vote_ms)),
                                                               "peaks_assoc": float(np.mean(rest_ms)),
                                                               "assoc": float(np.mean(assoc_ms))},
                              "peaks": int(counts[0]), "pairs": int(counts[1]), "tile": tile,
                              "band_split": band_split}), flush=True)
        return 0

    # ---- plain form (one launch sequence per event) on a 512-event sample,
    # median of five timed runs
    # (its own tile: one event per launch fills the GPU best with other tiles
    # than the batched step; autotuned on 64 events of the sample)
    plain_ctx = ht.Context(g, w.spec.layers)
    plain_ctx.set_option(ht.HT_OPT_MODE, ht.HT_MODE_PLAIN)
    if args.band_split is not None:
        plain_ctx.set_option(ht.HT_OPT_BAND_SPLIT, args.band_split)
    psub = batch.select(range(0, n_events, 8))
    if args.tile:
        for k, v in zip((ht.HT_OPT_TILE_PHI, ht.HT_OPT_TILE_D0, ht.HT_OPT_THREADS), args.tile.split(",")):
            plain_ctx.set_option(k, int(v))
    else:
        plain_ctx.autotune(ht.Hits.from_batch(psub.select(range(0, psub.n_events, 8)), device=dev))
    plain_tile = {"tile_phi": plain_ctx.get_option(ht.HT_OPT_TILE_PHI),
                  "tile_d0": plain_ctx.get_option(ht.HT_OPT_TILE_D0),
                  "threads": plain_ctx.get_option(ht.HT_OPT_THREADS),
                  "vote_items": plain_ctx.get_option(ht.HT_OPT_VOTE_ITEMS)}
    ph = ht.Hits.from_batch(psub, device=dev)
    pres = ht.Results(int(n_peaks * 0.2) + 4096, int(n_pairs * 0.2) + 65536, device=dev)
    plain_ctx.process(ph, w.threshold, w.window, pres, stream)
    plain_ctx.sync(allow_overflow=True)

    def plain_step():
        plain_ctx.process(ph, w.threshold, w.window, pres, stream)

    plain_ms, plain_runs = _median_ms(plain_step, stream, flush, 5)
    plain_ctx.sync(allow_overflow=True)
    plain_eps = psub.n_events / (plain_ms / 1e3)
    plain_ctx.close()
    del pres, ph

    # ---- serving: continuous batching at offered loads below and above capacity (rank 0, N=1)
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        from paper_1311_2769_gb300 import serve
        try:
            serving = serve.measure([2000.0, 5000.0, 10000.0, 13000.0, 20000.0, 50000.0], n_events=2000)
        except Exception as e:  # report, do not hide, a failing loop
            serving = {"error": f"{type(e).__name__}: {e}"}

    # ---- range voting against point voting (rank 0, N=1)
    range_vote = None
    if rank == 0 and world == 1 and not args.no_serving:
        try:
            range_vote = range_vote_report(dev)
        except Exception as e:  # report, do not hide, a failing measurement
            range_vote = {"error": f"{type(e).__name__}: {e}"}

    # ---- second Hough transform (rank 0, N=1)
    vertex = None
    if rank == 0 and world == 1 and not args.no_serving:
        try:
            vertex = vertex_report(dev)
        except Exception as e:
            vertex = {"error": f"{type(e).__name__}: {e}"}

    # ---- the dense event and the pileup batch (rank 0, N=1)
    secondary = None
    if rank == 0 and world == 1 and not args.no_serving:
        try:
            secondary = secondary_workloads(dev, stream, flush)
        except Exception as e:
            secondary = {"error": f"{type(e).__name__}: {e}"}

    # ---- rooflines of the two hot kernels: the method's FP32 work per
    # (hit, phi0, d0) cell (OPS_PER_CELL) against 152 SMs x 128 lanes x the
    # sampled clock; the dominant one (longer device time per step) is `roofline`
    peaks, peak_src = _peaks()
    clk = clocks.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    vote_s = float(np.mean(vote_ms)) / 1e3
    assoc_s = float(np.mean(assoc_ms)) / 1e3
    peak_tops = sms * 128 * sm_mhz * 1e6 / 1e12
    peak_basis = (f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (median SM clock under load); "
                  f"{OPS_PER_CELL} FP32 lane operations per (hit, phi0, d0) cell of the method: 8 arithmetic, "
                  f"1 IEEE division, 4 compare/convert")
    launches_per = max(1, waves)  # one launch of each kernel per wave
    per_launch_cells = hit_votes / launches_per
    vote_traffic = VOTE_DRAM_PER_HIT * n_hits / launches_per if VOTE_DRAM_PER_HIT else None
    assoc_traffic = ASSOC_DRAM_PER_HIT * n_hits / launches_per if ASSOC_DRAM_PER_HIT else None
    roof = {
        "vote_band_kernel": {"bound": "alu", "achieved": OPS_PER_CELL * hit_votes / vote_s / 1e12, "peak": peak_tops,
                             "unit": "TFLOP/s", "frac": OPS_PER_CELL * hit_votes / vote_s / 1e12 / peak_tops,
                             "traffic": vote_traffic, "kernel": "vote_band_kernel", "ops_per_cell": OPS_PER_CELL,
                             "cells_per_launch": per_launch_cells, "launches_per_step": launches_per,
                             "ms_per_launch": 1e3 * vote_s / launches_per, "peak_basis": peak_basis},
        "assoc_rec_kernel" if records else "assoc_kernel": {
            "bound": "alu", "achieved": OPS_PER_CELL * hit_votes / assoc_s / 1e12, "peak": peak_tops,
            "unit": "TFLOP/s", "frac": OPS_PER_CELL * hit_votes / assoc_s / 1e12 / peak_tops, "traffic": assoc_traffic,
            "kernel": "assoc_rec_kernel" if records else "assoc_kernel", "ops_per_cell": OPS_PER_CELL,
            "cells_per_launch": per_launch_cells, "launches_per_step": launches_per,
            "ms_per_launch": 1e3 * assoc_s / launches_per,
            "peak_basis": peak_basis + ("; the kernel decides every cell's association from the bins the vote "
                                        "recorded instead of binning again" if records else ""),
            "hbm": {"traffic_gbs": (assoc_traffic or 0.0) * launches_per / assoc_s / 1e9,
                    "peak_gbs": peaks.get("hbm_gbs"),
                    "frac": ((assoc_traffic or 0.0) * launches_per / assoc_s / 1e9) / peaks.get("hbm_gbs", 6800.0)}},
    }
    dom = max(roof, key=lambda k: roof[k]["ms_per_launch"])
    other = [k for k in roof if k != dom][0]
    ceilings = vote_ceilings(ht, g, batch, w, hit_votes, vote_s, vote_traffic * launches_per if vote_traffic else None,
                             peaks, dev) if rank == 0 else None
    acc_bytes = 4.0 * g.n_phi * g.n_d0 * g.n_kappa * n_events
    # the CPU leg after every GPU measurement: all cores, then one thread
    cpu = None
    single = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, batch)
        try:
            single = cpu_single_thread()
        except Exception as e:  # report, do not hide, a failing measurement
            single = {"error": f"{type(e).__name__}: {e}"}
        cpu["single_thread"] = single
    flips = None
    if single and "flip_fraction_plain_fp32" in single:
        flips = {"binary64_definition_gpu": 0.0,
                 "gpu_basis": "the bin is defined in binary64; the GPU reproduces it bit for bit (parity tests), "
                              "so its disagreement with an FP64 evaluation is 0",
                 "plain_fp32_context": single.pop("flip_fraction_plain_fp32"), "bound": 1e-5}
    line = {
        "metric": METRIC, "value": world * n_events / (ms / 1e3), "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "events_per_step": n_events, "hits_per_step": n_hits,
                   "grid": [g.n_phi, g.n_d0, g.n_kappa], "threshold": w.threshold, "window": w.window,
                   "mode": "batched persistent + CUDA graph", "l2": "flushed between timed steps",
                   "parallelism": f"events sharded, {world} independent rank(s)", "waves": waves,
                   "records": records, "band_split": band_split, **tile},
        "hit_votes_per_s": world * hit_votes / (ms / 1e3),
        "peaks_per_step": int(counts[0]), "pairs_per_step": int(counts[1]),
        "plain_events_per_s": plain_eps, "plain_runs_ms": plain_runs, "plain_stat": "median of 5",
        "plain_config": {"events": psub.n_events, "sample": "every 8th event of the batch", **plain_tile},
        "batched_over_plain": (n_events / (ms / 1e3)) / plain_eps,
        "phase_ms": {"vote": float(np.mean(vote_ms)), "peaks_assoc": float(np.mean(rest_ms)),
                     "assoc": float(np.mean(assoc_ms))},
        "roofline": roof[dom],
        f"roofline_{other.split('_kernel')[0]}": roof[other],
        "ceilings_vote": ceilings,
        "hbm": {"step_bytes_min": 2 * acc_bytes + 8.0 * n_hits,
                "achieved_gbs": (2 * acc_bytes + 8.0 * n_hits) / (ms / 1e3) / 1e9,
                "peak_gbs": peaks.get("hbm_gbs"), "peak_source": peak_src},
        "flip_fraction": flips,
        "clocks": clk,
        "gpu_launches": int(launches) * args.steps,
        "e2e": e2e,
        "secondary": secondary,
        "serving": serving,
        "range_vote": range_vote,
        "fit": fit_info,
        "merge": merge_info,
        "vertex": vertex,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--prune", type=int, default=None,
                    help="HT_OPT_PRUNE bits (1 vote, 2 association); default: the library's (3)")
    ap.add_argument("--workload", default=WORKLOAD, help="workload name (secondary lines use --no-extras)")
    ap.add_argument("--waves-of", type=int, default=0, help="admit accumulators for this many events at a time")
    ap.add_argument("--events", type=int, default=None, help="events per batch (default: the full 4096)")
    ap.add_argument("--tile", default="", help="vote tile 'phi,d0,threads' instead of autotuning")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed batched steps (no plain form, e2e or CPU baseline); for profiling")
    ap.add_argument("--hit-staging", type=int, default=None, help="HT_OPT_HIT_STAGING (default: the library's)")
    ap.add_argument("--host-chunks", type=int, default=0, help="HT_OPT_HOST_CHUNKS of the end-to-end pass")
    ap.add_argument("--vote-items", type=int, default=None, help="HT_OPT_VOTE_ITEMS (default: the library's)")
    ap.add_argument("--band-split", type=int, default=None, help="HT_OPT_BAND_SPLIT (default: the library's)")
    ap.add_argument("--record-budget-gb", type=float, default=160.0,
                    help="device memory for the vote records (GB); the 4096-event batch needs about 132")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
