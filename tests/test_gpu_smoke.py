"""The build/smoke entry point runs through the whole path on the GPU."""

import os
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_smoke_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import __graft_entry__
    __graft_entry__.smoke()
