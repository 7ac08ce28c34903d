"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/heart.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "heart.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:heart_status|const char \*)\s*(heart_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("heart_spectrometer_create", "heart_trace", "heart_submit", "heart_poll", "heart_last_error"):
        assert n in names


def test_library_builds_loads_and_exports_all_symbols():
    from paper_2503_16955_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    import paper_2503_16955_gb300 as H
    assert sorted(H.EXPORTS) == declared_functions()


def test_binding_structs_match_header_sizes():
    import paper_2503_16955_gb300 as H
    # sizes of the C structs as laid out by the header (x86-64 / aarch64 LP64)
    assert ctypes.sizeof(H.heart_tally) == 27 * 8
    assert ctypes.sizeof(H.heart_spectral_component) == 48
    assert ctypes.sizeof(H.heart_source_desc) == 8 + 8 + 24 + 24 + 8 + 16
    assert H.RECORD_DTYPE.itemsize == 112


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2503_16955_gb300 as H
    with pytest.raises(RuntimeError):
        H.library(str(tmp_path / "missing.so"))
