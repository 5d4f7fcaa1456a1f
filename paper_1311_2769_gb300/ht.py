"""Python binding of libht.so (argument marshalling only).

Every function here forwards to the C entry point of the same name declared
in ``include/ht.h``; all computation runs in the library's CUDA kernels.
Host inputs are numpy arrays, device inputs are CUDA tensors (PyTorch is used
for device memory and streams only).  If ``libht.so`` is missing the first
call raises: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libht.so")

HT_OK = 0
HT_ERR_INVALID_ARG = -1
HT_ERR_OOM = -2
HT_ERR_OVERFLOW = -3
HT_ERR_CUDA = -4
HT_ERR_TIMEOUT = -5
HT_ERR_BUDGET = -6
HT_ERR_STATE = -7

HT_HOST = 0
HT_DEVICE = 1

HT_OPT_MODE = 1
HT_OPT_TILE_PHI = 2
HT_OPT_TILE_D0 = 3
HT_OPT_THREADS = 4
HT_OPT_ACC_BUDGET = 5
HT_OPT_COUNT_STAGES = 6
HT_OPT_USE_GRAPH = 7
HT_OPT_PHASE_TIMING = 8
HT_OPT_LAUNCHES = 9
HT_OPT_ATILE_PHI = 10
HT_OPT_ATILE_D0 = 11
HT_OPT_PRUNE = 12
HT_OPT_VOTE_MODE = 13
HT_OPT_ASSOC_CURSORS = 14
HT_OPT_HOST_CHUNKS = 15
HT_OPT_ASSOC_INDEX = 16
HT_OPT_RECORDS = 17
HT_OPT_RECORD_BUDGET = 18
HT_OPT_WAVES = 19
HT_OPT_VOTE_ITEMS = 20
HT_OPT_HIT_STAGING = 21
HT_OPT_BAND_SPLIT = 22
HT_OPT_HOST_COPY = 23
HT_VOTE_POINT = 0
HT_VOTE_RANGE = 1
HT_VOTE_LINE = 2
HT_MODE_BATCHED = 0
HT_MODE_PLAIN = 1

EXPORTS = ("ht_create", "ht_destroy", "ht_set_option", "ht_get_option", "ht_vote", "ht_peaks",
           "ht_associate", "ht_process", "ht_get_accumulator", "ht_get_tables", "ht_sync",
           "ht_autotune", "ht_filter_stats", "ht_phase_times", "ht_peaks_noalloc", "ht_check_rcp", "ht_strerror", "ht_last_error",
           "ht_fit", "ht_vertices", "ht_merge", "ht_microbench")

PEAK_DTYPE = np.dtype([("event", np.int32), ("i_phi", np.int32), ("i_d0", np.int32),
                       ("i_kappa", np.int32), ("votes", np.uint32)])
VERTEX_DTYPE = np.dtype([("event", np.int32), ("i_x", np.int32), ("i_y", np.int32), ("votes", np.uint32)])
TRACK_DTYPE = np.dtype([("status", np.int32), ("n_hits", np.int32), ("cos_phi0", np.float64),
                        ("sin_phi0", np.float64), ("d0", np.float64), ("kappa", np.float64),
                        ("chi2", np.float64)])


class HtGeometry(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("layer_r", ctypes.c_void_p)]


class HtGrid(ctypes.Structure):
    _fields_ = [("n_phi", ctypes.c_int32), ("n_d0", ctypes.c_int32), ("n_kappa", ctypes.c_int32),
                ("d0_min", ctypes.c_float), ("d0_max", ctypes.c_float),
                ("kappa_min", ctypes.c_float), ("kappa_max", ctypes.c_float)]


class HtHits(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("layer", ctypes.c_void_p), ("event_offsets", ctypes.c_void_p),
                ("n_events", ctypes.c_int32), ("mem", ctypes.c_int32), ("n_hits", ctypes.c_int64)]


class HtResults(ctypes.Structure):
    _fields_ = [("peaks", ctypes.c_void_p), ("peak_cap", ctypes.c_int64),
                ("peak_offsets", ctypes.c_void_p), ("hit_idx", ctypes.c_void_p),
                ("pair_cap", ctypes.c_int64), ("counts", ctypes.c_void_p), ("mem", ctypes.c_int32)]


class HtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Load libht.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libht.so not found at {LIB_PATH}: build it with paper_1311_2769_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "ht_create": [P, P, P],
        "ht_destroy": [P],
        "ht_set_option": [P, i32, i64],
        "ht_get_option": [P, i32, P],
        "ht_vote": [P, P, P],
        "ht_peaks": [P, u32, P, i64, P],
        "ht_associate": [P, i32, P, P, i64, P],
        "ht_process": [P, P, u32, i32, P, P],
        "ht_get_accumulator": [P, i32, P],
        "ht_get_tables": [P, P, P, P],
        "ht_sync": [P],
        "ht_autotune": [P, P, P],
        "ht_filter_stats": [P, P, i32],
        "ht_phase_times": [P, P],
        "ht_check_rcp": [u32, u32, P],
        "ht_peaks_noalloc": [P, P, i32, u32, P, i64, P, P],
        "ht_fit": [P, P, P, i64, P],
        "ht_vertices": [P, P, P, u32, P, i64, P, P],
        "ht_merge": [P, P, P, i32, P, i64, P, P],
        "ht_microbench": [i32, i64, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.ht_strerror.argtypes = [ctypes.c_int]
    lib.ht_strerror.restype = ctypes.c_char_p
    lib.ht_last_error.argtypes = [P]
    lib.ht_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st: int, ctx=None, allow=()):
    if st == HT_OK or st in allow:
        return st
    lib = load()
    msg = lib.ht_strerror(st).decode()
    if ctx is not None:
        detail = lib.ht_last_error(ctx).decode()
        if detail:
            msg = f"{msg}: {detail}"
    raise HtError(st, msg)


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_device(a) -> bool:
    return a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _on_stream(stream):
    """Context in which torch allocates (and zero-fills) outputs on `stream`,
    so that the fill is ordered before the library's kernels on it."""
    import contextlib
    import torch
    if isinstance(stream, torch.cuda.Stream):
        return torch.cuda.stream(stream)
    if stream is not None:
        return torch.cuda.stream(torch.cuda.ExternalStream(int(stream)))
    return contextlib.nullcontext()


class Hits:
    """Keeps the arrays of an ``ht_hits`` alive while the library may read them."""

    def __init__(self, x, y, event_offsets, layer=None, z=None):
        dev = _is_device(x)
        if dev:
            import torch
            assert x.dtype == torch.float32 and y.dtype == torch.float32 and event_offsets.dtype == torch.int32
            x, y, event_offsets = x.contiguous(), y.contiguous(), event_offsets.contiguous()
            layer = None if layer is None else layer.contiguous()
            z = None if z is None else z.contiguous()
            n_events = int(event_offsets.numel()) - 1
            n_hits = int(x.numel())
        else:
            x = np.ascontiguousarray(x, dtype=np.float32)
            y = np.ascontiguousarray(y, dtype=np.float32)
            event_offsets = np.ascontiguousarray(event_offsets, dtype=np.int32)
            layer = None if layer is None else np.ascontiguousarray(layer, dtype=np.int8)
            z = None if z is None else np.ascontiguousarray(z, dtype=np.float32)
            n_events = event_offsets.shape[0] - 1
            n_hits = x.shape[0]
        self.arrays = (x, y, event_offsets, layer, z)
        self.struct = HtHits(_ptr(x), _ptr(y), _ptr(z), _ptr(layer), _ptr(event_offsets), n_events,
                             HT_DEVICE if dev else HT_HOST, n_hits)

    @classmethod
    def from_batch(cls, batch, device=None):
        """From a ``synth.Batch``; ``device='cuda'`` copies the arrays to the GPU first."""
        if device is None:
            return cls(batch.x, batch.y, batch.event_offsets, batch.layer, batch.z)
        import torch
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return cls(t(batch.x), t(batch.y), t(batch.event_offsets), t(batch.layer), t(batch.z))

    @property
    def n_events(self) -> int:
        return int(self.struct.n_events)

    @property
    def n_hits(self) -> int:
        return int(self.struct.n_hits)


# ---- C entry points, same names -------------------------------------------

def ht_create(grid, layer_r=()):
    lib = load()
    g = HtGrid(int(grid.n_phi), int(grid.n_d0), int(grid.n_kappa), float(grid.d0_min), float(grid.d0_max),
               float(grid.kappa_min), float(grid.kappa_max))
    lr = np.ascontiguousarray(layer_r, dtype=np.float32)
    geo = HtGeometry(lr.shape[0], lr.ctypes.data if lr.shape[0] else None)
    out = ctypes.c_void_p()
    _check(lib.ht_create(ctypes.byref(geo), ctypes.byref(g), ctypes.byref(out)))
    return out


def ht_destroy(ctx):
    return _check(load().ht_destroy(ctx))


def ht_set_option(ctx, key, value):
    return _check(load().ht_set_option(ctx, int(key), int(value)), ctx)


def ht_get_option(ctx, key) -> int:
    v = ctypes.c_int64()
    _check(load().ht_get_option(ctx, int(key), ctypes.byref(v)), ctx)
    return int(v.value)


def ht_vote(ctx, hits: Hits, stream=None):
    return _check(load().ht_vote(ctx, ctypes.byref(hits.struct), _stream_ptr(stream)), ctx)


def ht_peaks(ctx, threshold, cap=None):
    """Returns (peaks structured array, true count); grows the buffer to fit."""
    lib = load()
    n = ctypes.c_int64()
    cap = 1 << 16 if cap is None else int(cap)
    while True:
        out = np.empty(max(cap, 1), PEAK_DTYPE)
        st = lib.ht_peaks(ctx, int(threshold), out.ctypes.data, cap, ctypes.byref(n))
        if st == HT_ERR_OVERFLOW and n.value > cap:
            cap = int(n.value)
            continue
        _check(st, ctx)
        return out[: n.value].copy(), int(n.value)


def ht_associate(ctx, window, n_peaks, cap=None):
    """Returns (peak_offsets int64[n_peaks+1], hit_idx int32[n_pairs])."""
    lib = load()
    n = ctypes.c_int64()
    po = np.empty(int(n_peaks) + 1, np.int64)
    cap = 1 << 20 if cap is None else int(cap)
    while True:
        hi = np.empty(max(cap, 1), np.int32)
        st = lib.ht_associate(ctx, int(window), po.ctypes.data, hi.ctypes.data, cap, ctypes.byref(n))
        if st == HT_ERR_OVERFLOW and n.value > cap:
            cap = int(n.value)
            continue
        _check(st, ctx)
        return po, hi[: n.value].copy()


class Results:
    """Output buffers of ht_process (numpy on the host or CUDA tensors)."""

    def __init__(self, peak_cap, pair_cap, device=None):
        self.peak_cap, self.pair_cap = int(peak_cap), int(pair_cap)
        if device is None:
            self.peaks = np.zeros(max(self.peak_cap, 1), PEAK_DTYPE)
            self.peak_offsets = np.zeros(self.peak_cap + 1, np.int64)
            self.hit_idx = np.zeros(max(self.pair_cap, 1), np.int32)
            self.counts = np.zeros(2, np.int64)
            mem = HT_HOST
        else:
            import torch
            self.peaks = torch.zeros((max(self.peak_cap, 1), 5), dtype=torch.int32, device=device)
            self.peak_offsets = torch.zeros(self.peak_cap + 1, dtype=torch.int64, device=device)
            self.hit_idx = torch.zeros(max(self.pair_cap, 1), dtype=torch.int32, device=device)
            self.counts = torch.zeros(2, dtype=torch.int64, device=device)
            mem = HT_DEVICE
        self.struct = HtResults(_ptr(self.peaks), self.peak_cap, _ptr(self.peak_offsets), _ptr(self.hit_idx),
                                self.pair_cap, _ptr(self.counts), mem)

    def host(self):
        """(peaks structured array, peak_offsets, hit_idx) trimmed to the counts."""
        if isinstance(self.counts, np.ndarray):
            counts = self.counts
            pk, po, hi = self.peaks, self.peak_offsets, self.hit_idx
        else:
            counts = self.counts.cpu().numpy()
            pk = self.peaks.cpu().numpy().view(np.int32).reshape(-1, 5)
            pk = np.ascontiguousarray(pk).view(PEAK_DTYPE).reshape(-1)
            po, hi = self.peak_offsets.cpu().numpy(), self.hit_idx.cpu().numpy()
        np_, nq = min(int(counts[0]), self.peak_cap), min(int(counts[1]), self.pair_cap)
        return pk[:np_].copy(), po[: np_ + 1].copy(), hi[:nq].copy()


def ht_process(ctx, hits: Hits, threshold, window, results: Results, stream=None, allow_overflow=False):
    allow = (HT_ERR_OVERFLOW,) if allow_overflow else ()
    return _check(load().ht_process(ctx, ctypes.byref(hits.struct), int(threshold), int(window),
                                    ctypes.byref(results.struct), _stream_ptr(stream)), ctx, allow)


def ht_get_accumulator(ctx, event, shape):
    out = np.empty(shape, np.uint32)
    _check(load().ht_get_accumulator(ctx, int(event), out.ctypes.data), ctx)
    return out


def ht_get_tables(ctx, n_phi, n_d0):
    c = np.empty(n_phi, np.float32)
    s = np.empty(n_phi, np.float32)
    d = np.empty(n_d0, np.float32)
    _check(load().ht_get_tables(ctx, c.ctypes.data, s.ctypes.data, d.ctypes.data), ctx)
    return c, s, d


def ht_sync(ctx, allow_overflow=False):
    return _check(load().ht_sync(ctx), ctx, (HT_ERR_OVERFLOW,) if allow_overflow else ())


def ht_autotune(ctx, hits: Hits, stream=None):
    return _check(load().ht_autotune(ctx, ctypes.byref(hits.struct), _stream_ptr(stream)), ctx)


def ht_filter_stats(ctx, reset=False):
    out = np.zeros(4, np.int64)
    _check(load().ht_filter_stats(ctx, out.ctypes.data, 1 if reset else 0), ctx)
    return int(out[0]), int(out[1]), int(out[2])


def ht_phase_times(ctx):
    """(vote, peaks + association, whole step, association kernel) in ms."""
    ms = np.zeros(4, np.float32)
    _check(load().ht_phase_times(ctx, ms.ctypes.data), ctx)
    return float(ms[0]), float(ms[1]), float(ms[2]), float(ms[3])


def ht_peaks_noalloc(grid, acc, n_events, threshold, peaks, cap, count, stream=None):
    """Peaks of device accumulators with no device allocation (see ht.h).
    acc (uint32 or int32, at least n_events * cells elements), peaks (int32,
    at least 5 * cap elements) and count (int64) are contiguous CUDA tensors
    on the current device."""
    cells = int(grid.n_phi) * int(grid.n_d0) * int(grid.n_kappa)
    for name, t, dtypes, need in (("acc", acc, ("int32", "uint32"), int(n_events) * cells),
                                  ("peaks", peaks, ("int32",), 5 * int(cap)), ("count", count, ("int64",), 1)):
        if not getattr(t, "is_cuda", False) or not t.is_contiguous():
            raise ValueError(f"ht_peaks_noalloc: {name} must be a contiguous CUDA tensor")
        if str(t.dtype).replace("torch.", "") not in dtypes:
            raise ValueError(f"ht_peaks_noalloc: {name} must be {' or '.join(dtypes)}, not {t.dtype}")
        if t.numel() < need:
            raise ValueError(f"ht_peaks_noalloc: {name} holds {t.numel()} elements, {need} needed")
    g = HtGrid(int(grid.n_phi), int(grid.n_d0), int(grid.n_kappa), float(grid.d0_min), float(grid.d0_max),
               float(grid.kappa_min), float(grid.kappa_max))
    return _check(load().ht_peaks_noalloc(ctypes.byref(g), _ptr(acc), int(n_events), int(threshold), _ptr(peaks),
                                          int(cap), _ptr(count), _stream_ptr(stream)))


def ht_fit(ctx, results, cap=None, stream=None):
    """Circle fits of the candidates in `results` (see ht.h): a TRACK_DTYPE
    array for host results, else a CUDA uint8 tensor of cap * 48 bytes
    (tracks_host() reads it back)."""
    cap = results.peak_cap if cap is None else int(cap)
    if isinstance(results.counts, np.ndarray):
        n = int(min(results.counts[0], results.peak_cap, cap))
        out = np.zeros(max(n, 1), TRACK_DTYPE)
        _check(load().ht_fit(ctx, ctypes.byref(results.struct), out.ctypes.data, n, _stream_ptr(stream)), ctx)
        return out[:n]
    import torch
    with _on_stream(stream):
        out = torch.zeros(max(cap, 1) * TRACK_DTYPE.itemsize, dtype=torch.uint8, device=results.counts.device)
    _check(load().ht_fit(ctx, ctypes.byref(results.struct), _ptr(out), cap, _stream_ptr(stream)), ctx)
    return out


HT_MERGE_KEPT, HT_MERGE_DUPLICATE, HT_MERGE_BACKWARD, HT_MERGE_UNFITTED = 1, 0, -1, -2


def ht_merge(ctx, results, fits, radius=2, cap=None, stream=None):
    """Duplicate and mirror merging of fitted candidates (see ht.h).  Host
    results: (int32 state array, number kept).  Device results, with `fits`
    the device buffer ht_fit returned: (CUDA int32 state tensor, CUDA int64
    kept-count tensor)."""
    lib = load()
    if isinstance(results.counts, np.ndarray):
        n = int(min(results.counts[0], results.peak_cap, len(fits) if cap is None else int(cap)))
        f = np.ascontiguousarray(fits[:n], dtype=TRACK_DTYPE)
        state = np.zeros(max(n, 1), np.int32)
        kept = ctypes.c_int64()
        _check(lib.ht_merge(ctx, ctypes.byref(results.struct), f.ctypes.data, int(radius), state.ctypes.data, n,
                            ctypes.byref(kept), _stream_ptr(stream)), ctx)
        return state[:n], int(kept.value)
    import torch
    cap = results.peak_cap if cap is None else int(cap)
    assert fits.numel() >= cap * TRACK_DTYPE.itemsize, "fits buffer smaller than cap"
    dev = results.counts.device
    with _on_stream(stream):
        state = torch.zeros(max(cap, 1), dtype=torch.int32, device=dev)
        kept = torch.zeros(1, dtype=torch.int64, device=dev)
    _check(lib.ht_merge(ctx, ctypes.byref(results.struct), _ptr(fits), int(radius), _ptr(state), cap, _ptr(kept),
                        _stream_ptr(stream)), ctx)
    return state, kept


class HtVGrid(ctypes.Structure):
    _fields_ = [("n_x", ctypes.c_int32), ("n_y", ctypes.c_int32), ("x_min", ctypes.c_float),
                ("x_max", ctypes.c_float), ("y_min", ctypes.c_float), ("y_max", ctypes.c_float)]


def ht_vertices(ctx, vg, results, threshold, cap=None, stream=None):
    """Second Hough transform of the candidates in `results` (see ht.h).
    Host results: (VERTEX_DTYPE array, true count).  Device results: (CUDA
    uint8 tensor of cap * 16 bytes, CUDA int64 count tensor)."""
    v = HtVGrid(int(vg.n_x), int(vg.n_y), float(vg.x_min), float(vg.x_max), float(vg.y_min), float(vg.y_max))
    cap = 1 << 16 if cap is None else int(cap)
    lib = load()
    if isinstance(results.counts, np.ndarray):
        while True:
            out = np.zeros(max(cap, 1), VERTEX_DTYPE)
            n = ctypes.c_int64()
            st = lib.ht_vertices(ctx, ctypes.byref(v), ctypes.byref(results.struct), int(threshold), out.ctypes.data,
                                 cap, ctypes.byref(n), _stream_ptr(stream))
            if st == HT_ERR_OVERFLOW and n.value > cap:
                cap = int(n.value)
                continue
            _check(st, ctx)
            return out[: n.value].copy(), int(n.value)
    import torch
    dev = results.counts.device
    with _on_stream(stream):
        out = torch.zeros(max(cap, 1) * VERTEX_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    _check(lib.ht_vertices(ctx, ctypes.byref(v), ctypes.byref(results.struct), int(threshold), _ptr(out), cap,
                           _ptr(cnt), _stream_ptr(stream)), ctx)
    return out, cnt


def vertices_host(t, n):
    """The first n vertices of a device vertex buffer as a VERTEX_DTYPE array."""
    return np.frombuffer(t.cpu().numpy().tobytes(), VERTEX_DTYPE)[: int(n)].copy()


def tracks_host(t, n):
    """The first n fits of a device fit buffer as a TRACK_DTYPE array."""
    return np.frombuffer(t.cpu().numpy().tobytes(), TRACK_DTYPE)[: int(n)].copy()


HT_MB_FP32, HT_MB_SHARED_RED, HT_MB_FDIV, HT_MB_FP64 = 0, 1, 2, 3


def ht_microbench(kind, iters):
    """Measured throughput (operations/s) of one operation kind (see ht.h)."""
    rate = ctypes.c_double()
    _check(load().ht_microbench(int(kind), int(iters), ctypes.byref(rate)))
    return rate.value


def ht_check_rcp(first_bits, count):
    out = np.zeros(2, np.uint64)
    _check(load().ht_check_rcp(int(first_bits), int(count), out.ctypes.data))
    return int(out[0]), int(out[1])


class Context:
    """Owns one ht_ctx for a grid; thin sugar over the ht_* functions."""

    def __init__(self, grid, layer_r=()):
        self.grid = grid
        self.shape = (int(grid.n_phi), int(grid.n_d0), int(grid.n_kappa))
        self.handle = ht_create(grid, layer_r)
        self._hits = None

    def close(self):
        if self.handle:
            ht_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key, value):
        ht_set_option(self.handle, key, value)

    def get_option(self, key):
        return ht_get_option(self.handle, key)

    def vote(self, hits: Hits, stream=None):
        # device hits are borrowed: the later associate/fit/merge/vertices
        # calls read them, so the context keeps them alive until the next batch
        self._hits = hits
        ht_vote(self.handle, hits, stream)

    def peaks(self, threshold, cap=None):
        return ht_peaks(self.handle, threshold, cap)[0]

    def associate(self, window, n_peaks, cap=None):
        return ht_associate(self.handle, window, n_peaks, cap)

    def process(self, hits: Hits, threshold, window, results: Results, stream=None, allow_overflow=False):
        self._hits = hits  # borrowed device hits stay alive for fit/merge/vertices
        return ht_process(self.handle, hits, threshold, window, results, stream, allow_overflow)

    def accumulator(self, event=0):
        return ht_get_accumulator(self.handle, event, self.shape)

    def tables(self):
        return ht_get_tables(self.handle, self.shape[0], self.shape[1])

    def sync(self, allow_overflow=False):
        return ht_sync(self.handle, allow_overflow)

    def autotune(self, hits: Hits, stream=None):
        ht_autotune(self.handle, hits, stream)

    def filter_stats(self, reset=False):
        return ht_filter_stats(self.handle, reset)

    def phase_times(self):
        return ht_phase_times(self.handle)

    def fit(self, results, cap=None, stream=None):
        return ht_fit(self.handle, results, cap, stream)

    def merge(self, results, fits, radius=2, cap=None, stream=None):
        return ht_merge(self.handle, results, fits, radius, cap, stream)

    def vertices(self, vg, results, threshold, cap=None, stream=None):
        return ht_vertices(self.handle, vg, results, threshold, cap, stream)
