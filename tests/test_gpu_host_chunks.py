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
