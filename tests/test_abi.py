"""The C ABI library loads and exports every symbol include/rr.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rr_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2307_15412_gb300 import rr
    return ctypes.CDLL(rr.LIB_PATH)


def test_header_declares_boundary_calls():
    names = _declared()
    for must in ("rr_scene_upload", "rr_build_bvh", "rr_trace_frame", "rr_synth_if", "rr_range_doppler"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2307_15412_gb300 import rr
    assert sorted(rr.SIGNATURES) == _declared()


def test_version_callable_without_gpu(lib):
    lib.rr_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.rr_version()


def test_struct_layout_matches_header():
    from paper_2307_15412_gb300 import rr
    # doubles frame[9], tx[3], rx[8][3] = 36 doubles, 4 int32, 6 doubles
    assert ctypes.sizeof(rr.rr_radar) == 36 * 8 + 4 * 4 + 6 * 8
    assert ctypes.sizeof(rr.rr_raygrid) == 24
