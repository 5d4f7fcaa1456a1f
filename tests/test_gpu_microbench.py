"""The throughput microbenchmarks return plausible rates on the GPU and
reject bad arguments."""

import pytest

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


def test_microbench_rates(ht):
    p = torch.cuda.get_device_properties(0)
    lanes = p.multi_processor_count * 128
    fp32 = ht.ht_microbench(ht.HT_MB_FP32, 20000)
    # at most every FP32 lane at 2.5 GHz, at least a tenth of them at 0.5 GHz
    assert 0.1 * lanes * 0.5e9 < fp32 < lanes * 2.5e9, fp32
    red = ht.ht_microbench(ht.HT_MB_SHARED_RED, 5000)
    div = ht.ht_microbench(ht.HT_MB_FDIV, 5000)
    fp64 = ht.ht_microbench(ht.HT_MB_FP64, 2000)
    assert 0 < red < fp32 and 0 < div < fp32 and 0 < fp64 < fp32, (red, div, fp64, fp32)
    for kind, iters in ((4, 10), (-1, 10), (ht.HT_MB_FP32, 0)):
        with pytest.raises(ht.HtError) as ei:
            ht.ht_microbench(kind, iters)
        assert ei.value.status == ht.HT_ERR_INVALID_ARG
