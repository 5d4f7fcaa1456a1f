"""Host checks of the seeded input generator's batch packing (CPU only)."""

import numpy as np
import pytest

from paper_1311_2769_gb300 import synth


def test_concat_keeps_every_layer_id_valid():
    a = synth.generate(synth.WORKLOADS["single_event_10trk"], n_events=3)
    b = synth.generate(synth.WORKLOADS["batch_4096_lognormal"], n_events=2)
    for parts in ([a, b], [b, a]):
        c = synth.concat(parts)
        assert len(c.layer_r) == 13
        assert int(c.layer.max()) < len(c.layer_r) and int(c.layer.min()) >= 0
        assert c.n_events == 5 and c.event_offsets[-1] == c.n_hits
        assert np.all(np.diff(c.event_offsets) >= 0)
        assert np.array_equal(c.x[:parts[0].n_hits], parts[0].x)


def test_concat_rejects_different_layer_tables():
    a = synth.generate(synth.WORKLOADS["single_event_10trk"], n_events=1)
    b = synth.from_arrays(a.x, a.y, layer=a.layer, layer_r=np.asarray(a.layer_r) + 1.0)
    with pytest.raises(ValueError):
        synth.concat([a, b])
