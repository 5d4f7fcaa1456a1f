"""Host results copied wave by wave while later waves compute
(HT_OPT_HOST_CHUNKS) equal the device results, with and without output
overflow."""

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_2769_gb300 import build, ht as mod
    build.build()
    mod.load()
    return mod


def _stored(res):
    """Counts, the stored peaks, their row offsets, and the hits of the
    stored rows."""
    pk, po, hi = res.host()
    return [int(c) for c in np.asarray(res.counts)], pk, po, hi[: int(po[-1])] if len(po) else hi[:0]


def test_host_chunks_equal_device_results(ht):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=37, first_event=3)
    ctx = ht.Context(w.grid, w.spec.layers)
    dev = ht.Results(1 << 21, 1 << 26, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), w.threshold, 1, dev)
    ctx.sync()
    pk, po, hi = dev.host()
    assert len(pk) > 10000
    for chunks in (1, 4, 7, 64):
        ctx.set_option(ht.HT_OPT_HOST_CHUNKS, chunks)
        assert ctx.get_option(ht.HT_OPT_HOST_CHUNKS) == chunks
        for hits in (ht.Hits.from_batch(b), ht.Hits.from_batch(b, device="cuda")):
            rh = ht.Results(1 << 21, 1 << 26)
            ctx.process(hits, w.threshold, 1, rh)
            pk2, po2, hi2 = rh.host()
            assert np.array_equal(pk2, pk) and np.array_equal(po2, po) and np.array_equal(hi2, hi), chunks
    ctx.close()


def test_host_chunks_with_overflow(ht):
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=23, first_event=40)
    ctx = ht.Context(w.grid, w.spec.layers)
    full = ht.Results(1 << 21, 1 << 26)
    ctx.process(ht.Hits.from_batch(b), w.threshold, 1, full)
    pk, po, hi = full.host()
    for pcap, qcap in ((len(pk) // 3, 1 << 26), (1 << 21, int(po[len(pk) // 2]) + 5),
                       (len(pk) // 2, int(po[len(pk) // 4]) + 1)):
        want = None
        for chunks in (1, 3, 6):
            ctx.set_option(ht.HT_OPT_HOST_CHUNKS, chunks)
            rh = ht.Results(pcap, qcap)
            st = ctx.process(ht.Hits.from_batch(b), w.threshold, 1, rh, allow_overflow=True)
            assert st == ht.HT_ERR_OVERFLOW
            got = _stored(rh)
            if want is None:
                want = got
                n = min(len(pk), pcap)
                assert np.array_equal(got[1], pk[:n]) and np.array_equal(got[2], po[: n + 1])
                assert np.array_equal(got[3][: min(len(got[3]), qcap)], hi[: min(len(got[3]), qcap)])
            else:
                assert got[0] == want[0]
                for a, c in zip(got[1:], want[1:]):
                    assert np.array_equal(a, c), (pcap, qcap, chunks)
    with pytest.raises(ht.HtError) as ei:
        ctx.set_option(ht.HT_OPT_HOST_CHUNKS, 0)
    assert ei.value.status == ht.HT_ERR_INVALID_ARG
    ctx.close()


def _pinned_results(ht, pcap, qcap, shift=0):
    """Results in page-locked host memory; `shift` bytes past a 16-byte
    boundary (so the copy kernel takes its 4-byte or byte path)."""
    rh = ht.Results.__new__(ht.Results)
    rh.peak_cap, rh.pair_cap = pcap, qcap
    raw = [torch.empty(n + 16, dtype=torch.uint8).pin_memory() for n in (pcap * 20, (pcap + 1) * 8, qcap * 4, 16)]
    base = [r.data_ptr() + ((16 - r.data_ptr() % 16) % 16) + shift for r in raw[:3]] + [raw[3].data_ptr()]
    rh._raw = raw
    rh.struct = ht.HtResults(base[0], pcap, base[1], base[2], qcap, base[3], ht.HT_HOST)

    def host():
        import ctypes
        n = [int(v) for v in np.ctypeslib.as_array((ctypes.c_int64 * 2).from_address(base[3]))]
        npk = min(n[0], pcap)
        pk = np.ctypeslib.as_array((ctypes.c_int32 * (5 * npk)).from_address(base[0])).copy()
        po = np.ctypeslib.as_array((ctypes.c_int64 * (npk + 1)).from_address(base[1])).copy()
        nh = int(po[-1]) if npk else 0
        hi = np.ctypeslib.as_array((ctypes.c_int32 * max(nh, 1)).from_address(base[2]))[:nh].copy()
        return n, pk.view(ht.PEAK_DTYPE).reshape(-1) if npk else pk, po, hi
    rh.host = host
    return rh


@pytest.mark.parametrize("shift", [0, 4, 1])
def test_pinned_host_results_by_kernel_or_copy_engine(ht, shift):
    """Results copied into page-locked host memory by the copy kernel (32
    blocks, the default, or one) or by the copy engines equal the device
    results, for 1, 4 and 8 host chunks, at aligned and shifted destinations."""
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=29, first_event=11)
    ctx = ht.Context(w.grid, w.spec.layers)
    assert ctx.get_option(ht.HT_OPT_HOST_COPY) == 32
    dev = ht.Results(1 << 21, 1 << 26, device="cuda")
    ctx.process(ht.Hits.from_batch(b, device="cuda"), w.threshold, 1, dev)
    ctx.sync()
    pk, po, hi = dev.host()
    for copy in (32, 1, 0):
        ctx.set_option(ht.HT_OPT_HOST_COPY, copy)
        for chunks in (1, 4, 8):
            ctx.set_option(ht.HT_OPT_HOST_CHUNKS, chunks)
            rh = _pinned_results(ht, 1 << 21, 1 << 26, shift)
            ctx.process(ht.Hits.from_batch(b), w.threshold, 1, rh)
            n, pk2, po2, hi2 = rh.host()
            assert n == [len(pk), len(hi)]
            assert np.array_equal(pk2, pk) and np.array_equal(po2, po) and np.array_equal(hi2, hi), (copy, chunks)
    with pytest.raises(ht.HtError):
        ctx.set_option(ht.HT_OPT_HOST_COPY, -1)
    ctx.close()
