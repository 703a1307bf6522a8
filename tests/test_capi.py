"""Host-side checks of the C-ABI library: it builds for sm_103a, loads
without a GPU, and exports every entry point include/*.h declares. No
compute calls (no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(ss_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2303_10783_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_step_api():
    names = _declared()
    for n in ("ss_create_case", "ss_set_alloy", "ss_set_boundary", "ss_step", "ss_get_fields", "ss_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    lib, path = built_lib
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, "not exported by %s: %s" % (path, missing)


def test_struct_layouts_match_header(built_lib):
    """The ctypes mirrors agree with the header's field order (spot checks by size)."""
    from paper_2303_10783_gb300 import solid
    assert ctypes.sizeof(solid.Alloy) == 17 * 8
    assert ctypes.sizeof(solid.BC) == 8 + 8 + 8 + 8 + 8   # int (padded), h, Text, dTdt, int (padded)
    assert ctypes.sizeof(solid.Grid) == 4 * 4 + 3 * 8 + 8 + 8 + 16 + 8 + 8


def test_host_validation_without_gpu(built_lib):
    """Argument checks run on the host and return SS_EINVAL before touching the device."""
    from paper_2303_10783_gb300 import solid, cases
    lib = solid.load()
    g = solid.grid_struct(cases.cavity_2d(8, 6))
    n = ctypes.c_size_t()
    assert lib.ss_workspace_bytes(ctypes.byref(g), None) == solid.SS_EINVAL
    bad = solid.grid_struct(cases.cavity_2d(8, 6))
    bad.dim = 4
    assert lib.ss_workspace_bytes(ctypes.byref(bad), ctypes.byref(n)) == solid.SS_EINVAL
    assert b"dim" in lib.ss_last_error()
    bad = solid.grid_struct(cases.cavity_2d(8, 6))
    bad.dt = -1.0
    assert lib.ss_workspace_bytes(ctypes.byref(bad), ctypes.byref(n)) == solid.SS_EINVAL
    h = ctypes.c_void_p()
    assert lib.ss_create_case(ctypes.byref(g), None, 0, None, ctypes.byref(h)) == solid.SS_EINVAL
    assert lib.ss_step(None, 1) == solid.SS_EINVAL
    assert lib.ss_destroy(None) == solid.SS_OK
