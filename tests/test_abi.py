"""The C ABI library builds, loads without a GPU and exports every entry
point include/ht.h declares (no compute call is made here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ht.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ht_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1311_2769_gb300 import build, ht
    build.build()
    return ht.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ht_create", "ht_destroy", "ht_vote", "ht_peaks", "ht_associate", "ht_process",
                     "ht_get_accumulator", "ht_get_tables", "ht_sync", "ht_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1311_2769_gb300 import ht
    assert sorted(set(ht.EXPORTS)) == _declared()


def test_strerror_needs_no_gpu(lib):
    assert lib.ht_strerror(0) == b"ok"
    assert lib.ht_strerror(-3) == b"output capacity exceeded"
    assert lib.ht_strerror(12345) == b"unknown status"


def test_null_arguments_are_rejected_without_a_gpu(lib):
    assert lib.ht_destroy(None) == -1
    assert lib.ht_sync(None) == -1
    assert lib.ht_create(None, None, None) == -1


def test_argument_checks_of_the_extension_calls_need_no_gpu(lib):
    """Each of these rejects its arguments before any CUDA call."""
    rate = ctypes.c_double()
    for kind, iters in ((4, 10), (-1, 10), (0, 0)):
        assert lib.ht_microbench(kind, iters, ctypes.byref(rate)) == -1
    assert lib.ht_microbench(0, 10, None) == -1
    n = ctypes.c_int64()
    assert lib.ht_fit(None, None, None, 0, None) == -1
    assert lib.ht_merge(None, None, None, 2, None, 0, ctypes.byref(n), None) == -1
    assert lib.ht_vertices(None, None, None, 1, None, 0, ctypes.byref(n), None) == -1
    assert lib.ht_check_rcp(0, 0, None) == -1


def test_binding_option_numbers_match_the_header():
    from paper_1311_2769_gb300 import ht
    src = open(os.path.join(ROOT, "include", "ht.h")).read()
    opts = dict(re.findall(r"#define (HT_OPT_[A-Z0-9_]+) (\d+)", src))
    assert opts
    for name, value in opts.items():
        assert getattr(ht, name) == int(value), name
