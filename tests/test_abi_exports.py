"""The C-ABI library builds, loads on a machine without a GPU, and exports
every function that include/lbm.h and include/lbm3d.h declare (no compute
calls here)."""
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
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(lbm(?:3d)?_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1303_0107_gb300 import build
    path = build.build()
    return ctypes.CDLL(str(path))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lbm_create_geometry", "lbm_solve", "lbm_optimize_step", "lbm_read_fields",
                     "lbm3d_create", "lbm3d_solve", "lbm3d_optimize_step", "lbm3d_read_fields"):
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
    # server: configuration checks and the footprint rule are host-only
    srv = ctypes.c_void_p()
    bad = lib.ServerConfig(lib.F32, 0, 0, 100, 0)  # no slot
    assert L.lbm_server_create(ctypes.byref(bad), None, ctypes.byref(srv)) == 1 and not srv.value
    odd = lib.ServerConfig(lib.F32, 4, 0, 101, 0)  # odd tick
    assert L.lbm_server_create(ctypes.byref(odd), None, ctypes.byref(srv)) == 1
    L.lbm_server_destroy(None)
    assert L.lbm_server_cancel(None, 1) == 1
    L.lbm_debug_fail_alloc(-1)  # host-only switches
    L.lbm_debug_barrier_timeout(0)
    from paper_1303_0107_gb300 import lib3d
    L3 = lib3d._lib()
    h3 = ctypes.c_void_p()
    assert L3.lbm3d_create(None, None, None, ctypes.byref(h3)) == 1 and not h3.value
    L3.lbm3d_destroy(None)
    assert L3.lbm3d_set_block(None, 8) == 1
    k = ctypes.c_int32()
    assert L3.lbm3d_debug_task_counts(None, ctypes.byref(k), ctypes.byref(k)) == 1
    small = L.lbm_server_footprint(ctypes.byref(lib.make_params(128, 64, 0.8, 0.05)), 0)
    opt = L.lbm_server_footprint(ctypes.byref(lib.make_params(128, 64, 0.8, 0.05)), 5)
    half = L.lbm_server_footprint(ctypes.byref(lib.make_params(128, 64, 0.8, 0.05, precision=1)), 0)
    # FP32 populations alone are 9 * 64 * 128 * 4 bytes; optimising adds exchange scratch
    assert small > 9 * 64 * 128 * 4 and opt > small > half


def test_struct_layouts_match_header():
    from paper_1303_0107_gb300 import lib
    assert ctypes.sizeof(lib.Params) == 72
    assert ctypes.sizeof(lib.SolveResult) == 8 * 3 + 8 + 8 * 64 + 8 * 2 + 8 * 2
    assert ctypes.sizeof(lib.OptResult) == 16 + ctypes.sizeof(lib.SolveResult)


def test_struct_layouts_match_a_c_compiler(tmp_path):
    """sizeof and field offsets of the ABI structs as gcc lays them out from
    include/lbm.h, against the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    from paper_1303_0107_gb300 import lib, lib3d
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    checks = [("lbm_params", lib.Params, ["tau", "ports", "guard", "collision", "mirror", "c_smag"]),
              ("lbm_solve_result", lib.SolveResult, ["m_out", "fluid_cells"]),
              ("lbm_opt_result", lib.OptResult, ["solve"]),
              ("lbm_server_config", lib.ServerConfig, ["hbm_budget_bytes", "max_tick_steps"]),
              ("lbm_request", lib.Request, ["cell_types", "n_steps", "tag", "out_uy"]),
              ("lbm_served", lib.Served, ["t_done", "dp_first", "last"]),
              ("lbm_server_stats", lib.ServerStats, ["active", "busy_s", "budget_bytes"]),
              ("lbm_opt_plan", lib.OptPlan, ["tol", "patience", "reserved"]),
              ("lbm_opt_summary", lib.OptSummary, ["swapped", "dp_last"]),
              ("lbm3d_params", lib3d.Params3, ["precision", "tau", "u_max", "reinit", "collision", "c_smag",
                                               "mirror", "reserved"]),
              ("lbm3d_solve_result", lib3d.SolveResult3, ["n_outlets", "m_out", "fluid_cells"]),
              ("lbm3d_opt_result", lib3d.OptResult3, ["fluid_count", "solve"])]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', '#include "lbm3d.h"',
             "int main(void) {"]
    for cname, _, fields in checks:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = []
    for _, ct, fields in checks:
        want.append(ctypes.sizeof(ct))
        want += [getattr(ct, f).offset for f in fields]
    assert got == want
