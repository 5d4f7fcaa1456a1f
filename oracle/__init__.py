"""CPU oracle for the Hough-transform track finder — test infrastructure only.

Thin ctypes wrapper around ``libht_oracle.so`` (plain C, single-threaded,
binary64 arithmetic; see ``ht_oracle.c``).  Only the tests, the smoke check
and the bench's CPU-baseline leg may import this package.  It imports nothing
from the GPU library and the library imports nothing from it.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libht_oracle.so")
_SRC = os.path.join(_HERE, "ht_oracle.c")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction).  Returns the .so path."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ht_oracle.h"))):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Grid(ctypes.Structure):
    _fields_ = [("n_phi", ctypes.c_int32), ("n_d0", ctypes.c_int32), ("n_kappa", ctypes.c_int32),
                ("d0_min", ctypes.c_float), ("d0_max", ctypes.c_float),
                ("kappa_min", ctypes.c_float), ("kappa_max", ctypes.c_float)]


class VGrid(ctypes.Structure):
    _fields_ = [("n_x", ctypes.c_int32), ("n_y", ctypes.c_int32), ("x_min", ctypes.c_float),
                ("x_max", ctypes.c_float), ("y_min", ctypes.c_float), ("y_max", ctypes.c_float)]


PEAK_DTYPE = np.dtype([("event", np.int32), ("i_phi", np.int32), ("i_d0", np.int32),
                       ("i_kappa", np.int32), ("votes", np.uint32)])

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        G = ctypes.POINTER(Grid)
        f, i32, i64, u32 = ctypes.c_float, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        sig = {
            "hto_tables": (None, [G, P, P, P]),
            "hto_kbin": (i32, [G, f, f, i32, i32]),
            "hto_kbin_at": (i32, [G, f, f, f, f, f]),
            "hto_w64": (ctypes.c_double, [G, f, f, f, f, f]),
            "hto_kbin_fp32": (i32, [G, f, f, f, f, f]),
            "hto_w32": (f, [G, f, f, f, f, f]),
            "hto_kbin_cells": (None, [G, i64, P, P, P, P, P, P]),
            "hto_vote": (None, [G, P, P, P, i32, P]),
            "hto_vote_column": (None, [G, P, P, i64, i32, i32, P]),
            "hto_peaks": (i64, [G, P, i32, u32, P, i64]),
            "hto_is_peak": (i32, [G, P, u32, i32, i32, i32]),
            "hto_associate": (i64, [G, P, P, P, P, i64, i32, P, P, i64]),
            "hto_flip_count": (None, [G, P, P, P, i32, P]),
            "hto_run_events": (None, [G, P, P, P, i32, u32, i32, i32, P]),
            "hto_edges": (None, [G, P, P, P]),
            "hto_code_at": (i32, [G, f, f, f, f, f]),
            "hto_code_cells": (None, [G, i64, P, P, P, P, P, P]),
            "hto_range": (i32, [G, f, f, i32, i32, P, P]),
            "hto_vote_range": (None, [G, P, P, P, i32, P]),
            "hto_associate_range": (i64, [G, P, P, P, P, i64, i32, P, P, i64]),
            "hto_fit": (None, [G, P, P, P, i64, P, P, P]),
            "hto_fit_row": (None, [G, P, P, P, i64, i32, P]),
            "hto_vertex_vote": (None, [G, ctypes.POINTER(VGrid), P, i64, i32, P]),
            "hto_vertex_peaks": (i64, [ctypes.POINTER(VGrid), P, i32, u32, P, i64]),
            "hto_line_bin": (i32, [G, f, f, i32]),
            "hto_vote_line": (None, [G, P, P, P, i32, P]),
            "hto_associate_line": (i64, [G, P, P, P, P, i64, i32, P, P, i64]),
            "hto_merge": (i64, [G, P, P, P, i64, P, P, P, i32, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def grid_struct(g) -> Grid:
    """Accepts any object with the seven grid attributes (e.g. synth.Grid)."""
    return Grid(int(g.n_phi), int(g.n_d0), int(g.n_kappa), float(g.d0_min), float(g.d0_max),
                float(g.kappa_min), float(g.kappa_max))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _offs(event_offsets, n):
    if event_offsets is None:
        return np.array([0, n], dtype=np.int32)
    return np.ascontiguousarray(event_offsets, dtype=np.int32)


def tables(g):
    gs = grid_struct(g)
    c = np.empty(gs.n_phi, np.float32)
    s = np.empty(gs.n_phi, np.float32)
    d = np.empty(gs.n_d0, np.float32)
    lib().hto_tables(ctypes.byref(gs), _ptr(c), _ptr(s), _ptr(d))
    return c, s, d


def kbin(g, x, y, i, j) -> int:
    return int(lib().hto_kbin(ctypes.byref(grid_struct(g)), float(x), float(y), int(i), int(j)))


def kbin_at(g, x, y, c, s, d) -> int:
    return int(lib().hto_kbin_at(ctypes.byref(grid_struct(g)), float(x), float(y), float(c), float(s), float(d)))


def w64(g, x, y, c, s, d) -> float:
    return float(lib().hto_w64(ctypes.byref(grid_struct(g)), float(x), float(y), float(c), float(s), float(d)))


def kbin_cells(g, x, y, c, s, d) -> np.ndarray:
    """Vectorised kbin_at over equal-length arrays."""
    gs = grid_struct(g)
    x, y, c, s, d = (_f32(v) for v in (x, y, c, s, d))
    out = np.empty(x.shape[0], np.int32)
    lib().hto_kbin_cells(ctypes.byref(gs), x.shape[0], _ptr(x), _ptr(y), _ptr(c), _ptr(s), _ptr(d), _ptr(out))
    return out


def kbin_fp32(g, x, y, c, s, d) -> int:
    return int(lib().hto_kbin_fp32(ctypes.byref(grid_struct(g)), float(x), float(y), float(c), float(s), float(d)))


def w32(g, x, y, c, s, d) -> float:
    """The float32 op-order bin coordinate (NaN when den <= 0)."""
    return float(lib().hto_w32(ctypes.byref(grid_struct(g)), float(x), float(y), float(c), float(s), float(d)))


def vote(g, x, y, event_offsets=None) -> np.ndarray:
    """Accumulators [n_events, n_phi, n_d0, n_kappa] uint32."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    offs = _offs(event_offsets, x.shape[0])
    ne = offs.shape[0] - 1
    acc = np.empty((ne, gs.n_phi, gs.n_d0, gs.n_kappa), dtype=np.uint32)
    lib().hto_vote(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(offs), ne, _ptr(acc))
    return acc


def vote_column(g, x, y, i, j) -> np.ndarray:
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    out = np.empty(gs.n_kappa, np.uint32)
    lib().hto_vote_column(ctypes.byref(gs), _ptr(x), _ptr(y), x.shape[0], int(i), int(j), _ptr(out))
    return out


def peaks(g, acc, threshold) -> np.ndarray:
    """Structured array of (event, i_phi, i_d0, i_kappa, votes), ascending."""
    gs = grid_struct(g)
    acc = np.ascontiguousarray(acc, dtype=np.uint32)
    ne = acc.shape[0]
    cap = 1024
    while True:
        out = np.empty(cap, PEAK_DTYPE)
        n = lib().hto_peaks(ctypes.byref(gs), _ptr(acc), ne, int(threshold), _ptr(out), cap)
        if n <= cap:
            return out[:n].copy()
        cap = n


def is_peak(g, acc1, threshold, i, j, k) -> bool:
    gs = grid_struct(g)
    acc1 = np.ascontiguousarray(acc1, dtype=np.uint32)
    return bool(lib().hto_is_peak(ctypes.byref(gs), _ptr(acc1), int(threshold), int(i), int(j), int(k)))


def associate(g, x, y, event_offsets, pk, window):
    """CSR (peak_offsets int64[n_peaks+1], hit_idx int32[n_pairs])."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    offs = _offs(event_offsets, x.shape[0])
    pk = np.ascontiguousarray(pk, dtype=PEAK_DTYPE)
    po = np.empty(pk.shape[0] + 1, np.int64)
    cap = 1 << 16
    while True:
        hi = np.empty(cap, np.int32)
        n = lib().hto_associate(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(offs), _ptr(pk), pk.shape[0],
                                int(window), _ptr(po), _ptr(hi), cap)
        if n <= cap:
            return po, hi[:n].copy()
        cap = n


def flip_count(g, x, y, event_offsets=None):
    """(binary64 votes, float32 votes, columns whose bins differ)."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    offs = _offs(event_offsets, x.shape[0])
    out = np.zeros(3, np.int64)
    lib().hto_flip_count(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(offs), offs.shape[0] - 1, _ptr(out))
    return int(out[0]), int(out[1]), int(out[2])


def run_events(g, x, y, event_offsets, threshold, window, n_threads):
    """Whole path per event on n_threads host threads: (votes, peaks, pairs)."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    offs = _offs(event_offsets, x.shape[0])
    out = np.zeros(3, np.int64)
    lib().hto_run_events(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(offs), offs.shape[0] - 1,
                         int(threshold), int(window), int(n_threads), _ptr(out))
    return int(out[0]), int(out[1]), int(out[2])


# ---- range voting --------------------------------------------------------

UNDEF = -2  # corner code when the corner's denominator is not positive


def edges(g):
    """(cos, sin) of the phi0 edges m 2pi/n_phi and the n_d0 + 1 d0 edges (float32)."""
    gs = grid_struct(g)
    c = np.empty(gs.n_phi, np.float32)
    s = np.empty(gs.n_phi, np.float32)
    d = np.empty(gs.n_d0 + 1, np.float32)
    lib().hto_edges(ctypes.byref(gs), _ptr(c), _ptr(s), _ptr(d))
    return c, s, d


def code_at(g, x, y, c, s, d) -> int:
    return int(lib().hto_code_at(ctypes.byref(grid_struct(g)), float(x), float(y), float(c), float(s), float(d)))


def code_cells(g, x, y, c, s, d) -> np.ndarray:
    """Corner codes (UNDEF, -1 below, n_kappa above, else the bin) over equal-length arrays."""
    gs = grid_struct(g)
    x, y, c, s, d = (_f32(v) for v in (x, y, c, s, d))
    out = np.empty(x.shape[0], np.int32)
    lib().hto_code_cells(ctypes.byref(gs), x.shape[0], _ptr(x), _ptr(y), _ptr(c), _ptr(s), _ptr(d), _ptr(out))
    return out


def range_of(g, x, y, i, j):
    """(lo, hi) bins hit (x, y) votes for in cell (i, j) under range voting, or None."""
    lo = ctypes.c_int32()
    hi = ctypes.c_int32()
    ok = lib().hto_range(ctypes.byref(grid_struct(g)), float(x), float(y), int(i), int(j),
                         ctypes.byref(lo), ctypes.byref(hi))
    return (lo.value, hi.value) if ok else None


def vote_range(g, x, y, event_offsets=None) -> np.ndarray:
    """Range-vote accumulators [n_events, n_phi, n_d0, n_kappa] uint32."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    offs = _offs(event_offsets, x.shape[0])
    ne = offs.shape[0] - 1
    acc = np.empty((ne, gs.n_phi, gs.n_d0, gs.n_kappa), dtype=np.uint32)
    lib().hto_vote_range(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(offs), ne, _ptr(acc))
    return acc


def associate_range(g, x, y, event_offsets, pk, window):
    """Range association CSR (peak_offsets int64[n_peaks+1], hit_idx int32[n_pairs])."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    offs = _offs(event_offsets, x.shape[0])
    pk = np.ascontiguousarray(pk, dtype=PEAK_DTYPE)
    po = np.empty(pk.shape[0] + 1, np.int64)
    cap = 1 << 16
    while True:
        hi = np.empty(cap, np.int32)
        n = lib().hto_associate_range(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(offs), _ptr(pk), pk.shape[0],
                                      int(window), _ptr(po), _ptr(hi), cap)
        if n <= cap:
            return po, hi[:n].copy()
        cap = n


# ---- circle fit ------------------------------------------------------------

TRACK_DTYPE = np.dtype([("status", np.int32), ("n_hits", np.int32), ("cos_phi0", np.float64),
                        ("sin_phi0", np.float64), ("d0", np.float64), ("kappa", np.float64),
                        ("chi2", np.float64)])


def fit(g, x, y, pk, peak_offsets, hit_idx) -> np.ndarray:
    """Circle fit of every candidate's CSR row: structured array TRACK_DTYPE."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    pk = np.ascontiguousarray(pk, dtype=PEAK_DTYPE)
    po = np.ascontiguousarray(peak_offsets, dtype=np.int64)
    hi = np.ascontiguousarray(hit_idx, dtype=np.int32)
    out = np.zeros(pk.shape[0], TRACK_DTYPE)
    lib().hto_fit(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(pk), pk.shape[0], _ptr(po), _ptr(hi), _ptr(out))
    return out


def fit_hits(g, x, y, i_kappa) -> np.void:
    """Circle fit of the given hits (all of them, in order) for a peak in kappa bin i_kappa."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    idx = np.arange(x.shape[0], dtype=np.int32)
    out = np.zeros(1, TRACK_DTYPE)
    lib().hto_fit_row(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(idx), x.shape[0], int(i_kappa), _ptr(out))
    return out[0]


MERGE_KEPT, MERGE_DUPLICATE, MERGE_BACKWARD, MERGE_UNFITTED = 1, 0, -1, -2


def merge(g, x, y, pk, peak_offsets, hit_idx, fits, radius=2):
    """Duplicate and mirror merging of fitted candidates: (state int32 per
    candidate, number kept)."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    pk = np.ascontiguousarray(pk, dtype=PEAK_DTYPE)
    po = np.ascontiguousarray(peak_offsets, dtype=np.int64)
    hi = np.ascontiguousarray(hit_idx, dtype=np.int32)
    fits = np.ascontiguousarray(fits, dtype=TRACK_DTYPE)
    assert fits.shape[0] == pk.shape[0] and po.shape[0] == pk.shape[0] + 1
    state = np.zeros(pk.shape[0], np.int32)
    kept = lib().hto_merge(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(pk), pk.shape[0], _ptr(po), _ptr(hi),
                           _ptr(fits), int(radius), _ptr(state))
    return state, int(kept)


# ---- second Hough transform: displaced vertices ------------------------------

VERTEX_DTYPE = np.dtype([("event", np.int32), ("i_x", np.int32), ("i_y", np.int32), ("votes", np.uint32)])


def vgrid_struct(v) -> VGrid:
    """Any object with n_x, n_y, x_min, x_max, y_min, y_max."""
    return VGrid(int(v.n_x), int(v.n_y), float(v.x_min), float(v.x_max), float(v.y_min), float(v.y_max))


def vertex_vote(g, v, pk, n_events) -> np.ndarray:
    """Vertex accumulators [n_events, n_x, n_y] uint32 from the candidates pk."""
    gs, vs = grid_struct(g), vgrid_struct(v)
    pk = np.ascontiguousarray(pk, dtype=PEAK_DTYPE)
    acc = np.empty((int(n_events), vs.n_x, vs.n_y), np.uint32)
    lib().hto_vertex_vote(ctypes.byref(gs), ctypes.byref(vs), _ptr(pk), pk.shape[0], int(n_events), _ptr(acc))
    return acc


def vertex_peaks(v, acc, threshold) -> np.ndarray:
    vs = vgrid_struct(v)
    acc = np.ascontiguousarray(acc, dtype=np.uint32)
    cap = 1024
    while True:
        out = np.empty(cap, VERTEX_DTYPE)
        n = lib().hto_vertex_peaks(ctypes.byref(vs), _ptr(acc), acc.shape[0], int(threshold), _ptr(out), cap)
        if n <= cap:
            return out[:n].copy()
        cap = n


# ---- straight displaced tracks (kappa = 0) -----------------------------------

def line_bin(g, x, y, i) -> int:
    return int(lib().hto_line_bin(ctypes.byref(grid_struct(g)), float(x), float(y), int(i)))


def vote_line(g, x, y, event_offsets=None) -> np.ndarray:
    """Line-vote accumulators [n_events, n_phi, n_d0, 1] uint32 (grid with n_kappa = 1)."""
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    offs = _offs(event_offsets, x.shape[0])
    ne = offs.shape[0] - 1
    acc = np.empty((ne, gs.n_phi, gs.n_d0, 1), dtype=np.uint32)
    lib().hto_vote_line(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(offs), ne, _ptr(acc))
    return acc


def associate_line(g, x, y, event_offsets, pk, window):
    gs = grid_struct(g)
    x, y = _f32(x), _f32(y)
    offs = _offs(event_offsets, x.shape[0])
    pk = np.ascontiguousarray(pk, dtype=PEAK_DTYPE)
    po = np.empty(pk.shape[0] + 1, np.int64)
    cap = 1 << 16
    while True:
        hi = np.empty(cap, np.int32)
        n = lib().hto_associate_line(ctypes.byref(gs), _ptr(x), _ptr(y), _ptr(offs), _ptr(pk), pk.shape[0],
                                     int(window), _ptr(po), _ptr(hi), cap)
        if n <= cap:
            return po, hi[:n].copy()
        cap = n
