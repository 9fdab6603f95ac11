"""The C-ABI library loads and exports every entry point of include/gs.h; host
argument checks answer without touching a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2507_04004_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    B.build()
    from paper_2507_04004_b300 import _native
    return _native


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_are_exported(native):
    lib = native.lib()
    names = _declared()
    assert "gs_project" in names and "gs_render_bwd" in names and len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(native.EXPORTED) == set(names)


def test_version_and_status_strings(native):
    assert native.gs_version().startswith("gsb300")
    assert native.status_str(native.GS_ERR_CAPACITY) == "pair buffer too small"


def test_workspace_size_and_layout(native):
    f = native.gs_frame(4, 1920, 1080)
    size = native.gs_workspace_size(1_000_000, f, 1 << 24)
    L = native.gs_workspace_layout(1_000_000, f, 1 << 24)
    assert size == L.total and size > 0
    offs = [getattr(L, k) for k, _ in native.gs_layout._fields_ if k != "total"]
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    assert L.rects - L.records == 4 * 1_000_000 * 48
    # invalid geometry
    assert native.gs_workspace_size(0, f, 100) == 0
    assert native.gs_workspace_size(10, native.gs_frame(1, 0, 10), 100) == 0
    assert native.gs_workspace_size(10, native.gs_frame(1, 9000, 10), 100) == 0
    assert native.gs_workspace_size(10, f, 0) == 0


def test_argument_errors_return_synchronously(native):
    lib = native.lib()
    f = native.gs_frame(1, 64, 48)
    ws = native.gs_workspace(None, 10, 100, f)
    cfg = native.gs_config(1 / 255, 0.99, 1e-4, 0.2, 0.3, 1.3)
    m = native.gs_map(10, 0, 0, None, None, None, None, None, None)
    # null workspace pointer
    assert lib.gs_project(C.byref(m), None, C.byref(cfg), C.byref(ws), None) == native.GS_ERR_ARG
    assert lib.gs_bin_sort(C.byref(ws), None) == native.GS_ERR_ARG
    # misaligned workspace pointer, null map arrays, bad SH degree, bad config
    ws.ptr = 0x1000 + 8
    assert lib.gs_bin_sort(C.byref(ws), None) == native.GS_ERR_ARG
    ws.ptr = 0x1000
    assert lib.gs_project(C.byref(m), C.c_void_p(0x2000), C.byref(cfg), C.byref(ws), None) == native.GS_ERR_ARG
    m2 = native.gs_map(10, 4, 0, 0x1000, 0x1000, 0x1000, 0x1000, 0x1000, 0x1000)
    assert lib.gs_project(C.byref(m2), C.c_void_p(0x2000), C.byref(cfg), C.byref(ws), None) == native.GS_ERR_ARG
    m3 = native.gs_map(11, 0, 0, 0x1000, 0x1000, 0x1000, 0x1000, 0x1000, None)
    assert lib.gs_project(C.byref(m3), C.c_void_p(0x2000), C.byref(cfg), C.byref(ws), None) == native.GS_ERR_ARG
    bad = native.gs_config(0.0, 0.99, 1e-4, 0.2, 0.3, 1.3)
    m4 = native.gs_map(10, 0, 0, 0x1000, 0x1000, 0x1000, 0x1000, 0x1000, None)
    assert lib.gs_project(C.byref(m4), C.c_void_p(0x2000), C.byref(bad), C.byref(ws), None) == native.GS_ERR_ARG
    assert lib.gs_render_fwd(C.byref(cfg), C.byref(ws), None, None, None, None, None, None) == native.GS_ERR_ARG
    assert lib.gs_pose_jacobian(C.byref(m4), C.c_void_p(0x2000), C.byref(cfg), C.byref(ws), None, 0, None, None,
                                None) == native.GS_ERR_ARG
