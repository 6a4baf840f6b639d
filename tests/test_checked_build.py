"""The bounds-checked build (paper_1303_0107_gb300.build.build(checked=True),
loaded with LBM_CHECKED=1): every population, field and mask access of the
step and reduction kernels is checked against its allocation (a violation is
printed and skipped), and canary blocks on both sides of each lattice's
population planes are checked after every solve and optimiser step.

Run in a child process (the binding loads one library per process): a solve
and an exchange on the 128 x 64 T-junction, and on the 72 x 34 x 34 D3Q19
tree with and without packed cell tasks, report no violation; after the
test hook overwrites part of a canary (a host-side memset inside the
allocation: no device fault) the next solve fails with LBM_ERR_CUDA naming
the canary.  The normal build has no canaries and refuses the hook.
"""
import os
import subprocess
import sys

import pytest

import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = """
import sys
sys.path.insert(0, {root!r})
import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I
cfg = I.config_t_junction()
lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"])
lat.solve(400)
lat.optimize_step(3, 200)
import os
c3 = I.config_tree3d_small()
for pb in ("24", "32"):  # the D3Q19 step on row segments and packed cells, through an exchange
    os.environ["LBM3D_PACK_BELOW"] = pb
    l3 = L.Lattice3(c3["cells"], c3["tau"], c3["u_max"])
    l3.solve(100)
    l3.optimize_step(10, 100)
    l3.close()
print("SOLVED", flush=True)
lat.debug_damage_canary()
try:
    lat.solve(2)
    print("NOT DETECTED")
except L.LbmError as e:
    print("DETECTED", e.status, str(e))
"""


def test_checked_build_finds_a_damaged_canary():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_0107_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, LBM_CHECKED="1")
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "SOLVED" in out.stdout, out.stdout[-2000:]
    assert "lbm bounds" not in out.stdout  # no access outside its allocation
    assert "DETECTED 4" in out.stdout and "canary" in out.stdout, out.stdout[-2000:]


def test_normal_build_has_no_canaries():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load_library()
    cfg = I.config_t_junction()
    lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"])
    with pytest.raises(L.LbmError) as e:
        lat.debug_damage_canary()
    assert e.value.status == 1
    lat.close()
