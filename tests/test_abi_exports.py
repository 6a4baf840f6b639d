"""The C-ABI library builds, loads on a machine without a GPU, and exports
every function that include/lbm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(lbm_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1303_0107_gb300 import build
    path = build.build()
    return ctypes.CDLL(str(path))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lbm_create_geometry", "lbm_solve", "lbm_optimize_step", "lbm_read_fields"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in _declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_host_only_entry_points(built_lib):
    from paper_1303_0107_gb300 import lib
    L = lib.load_library()
    assert L.lbm_status_str(0) == b"ok"
    assert L.lbm_bytes_per_fluid_update(lib.F32) == pytest.approx(72.125)
    assert L.lbm_bytes_per_fluid_update(lib.BF16_SHIFTED) == pytest.approx(36.125)
    # argument checks run before any CUDA call
    h = ctypes.c_void_p()
    assert L.lbm_create_geometry(None, None, None, ctypes.byref(h)) == 1
    assert not h.value
    L.lbm_destroy(None)


def test_struct_layouts_match_header():
    from paper_1303_0107_gb300 import lib
    assert ctypes.sizeof(lib.Params) == 56
    assert ctypes.sizeof(lib.SolveResult) == 8 * 3 + 8 + 8 * 64 + 8 * 2 + 8 * 2
    assert ctypes.sizeof(lib.OptResult) == 16 + ctypes.sizeof(lib.SolveResult)
