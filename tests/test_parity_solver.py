"""GPU solver vs the FP64 oracle, through the C ABI.

Tolerance (FP32 storage, stated for the hot path): max-norm error relative to
the max-norm of the oracle field <= 1e-5 for rho - rho0, u_x, u_y, and
relative error <= 1e-5 on the pressure drop and the outlet flow rates.
After an even number of steps the GPU's stored populations are the
post-collision state, the same quantity the oracle keeps, so they are
compared directly (FP32 rounding per step: 2e-6 of the population scale).
"""
import numpy as np
import pytest

import paper_1303_0107_gb300 as L
from paper_1303_0107_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load_library()


def _run_both(ora, cells, tau, u_max, steps, outlet=0, residual_every=0):
    ny, nx = cells.shape
    lat = L.Lattice(cells, tau, u_max, outlet=outlet, residual_every=residual_every)
    g = lat.solve(steps)
    p = ora.make_params(nx, ny, tau, 1.0, u_max, outlet)
    s = ora.Solver(p, cells, residual_every=residual_every)
    o = s.solve(steps)
    return lat, g, s, o


def _rel_inf(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def _check_fields(lat, s, cells, tol=TOL):
    fluid = cells == 0
    drho = lat.read(L.FIELD_DRHO)
    ux = lat.read(L.FIELD_UX)
    uy = lat.read(L.FIELD_UY)
    ref_drho = (s.rho - 1.0) * fluid
    assert _rel_inf(drho, ref_drho) <= tol
    assert _rel_inf(ux, s.ux) <= tol
    if np.abs(s.uy).max() > 1e-12:
        assert np.abs(uy - s.uy).max() <= tol * max(np.abs(s.ux).max(), np.abs(s.uy).max())
    rho = lat.read(L.FIELD_RHO)
    assert np.all(rho[~fluid] == 0) and np.all(ux[~fluid] == 0) and np.all(uy[~fluid] == 0)
    assert np.abs(rho - s.rho).max() <= 2e-7 * 4


def _check_pops(lat, s, cells, tol=4e-6):
    g = lat.read(L.FIELD_POPS)  # shifted post-collision populations
    f_gpu = g.astype(np.float64) + W[:, None, None] * 1.0
    fluid = cells == 0
    err = np.abs(f_gpu - s.f)[:, fluid].max()
    assert err <= tol * W.max(), err


@pytest.mark.parametrize("steps", [2, 4, 6, 10])
def test_first_steps_tiny_channel(ora, steps):
    cells = I.channel(16, 6)
    lat, g, s, o = _run_both(ora, cells, 0.8, 0.05, steps)
    _check_pops(lat, s, cells)
    _check_fields(lat, s, cells, tol=2e-6)


@pytest.mark.parametrize("shape,seed", [((34, 10), 1), ((64, 20), 2), ((100, 40), 3), ((70, 31), 4)])
def test_irregular_walls_ragged_sizes(ora, shape, seed):
    """Random obstacles exercise bounce-back in every direction; sizes that are
    not multiples of the 32-cell tile leave ragged row segments."""
    nx, ny = shape
    cells = I.random_blobs(nx, ny, seed, density=0.2)
    lat, g, s, o = _run_both(ora, cells, 0.7, 0.03, 40)
    _check_pops(lat, s, cells, tol=2e-5)
    _check_fields(lat, s, cells)
    assert abs(g["dp"] - o["dp"]) <= TOL * abs(o["dp"])


@pytest.mark.parametrize("outlet", [0, 1])
def test_t_junction_full_solve(ora, outlet):
    cfg = I.config_t_junction()
    lat, g, s, o = _run_both(ora, cfg["cells"], cfg["tau"], cfg["u_max"], cfg["steps"], outlet=outlet,
                             residual_every=100)
    _check_fields(lat, s, cfg["cells"])
    assert abs(g["dp"] - o["dp"]) <= TOL * abs(o["dp"])
    assert abs(g["m_in"] - o["m_in"]) <= TOL * abs(o["m_in"])
    assert g["n_outlets"] == len(o["m_out"]) == 2
    assert np.abs(g["m_out"] - o["m_out"]).max() <= TOL * np.abs(o["m_out"]).max()
    assert g["theta"] == pytest.approx(o["theta"], rel=TOL)
    assert abs(g["dg"] - o["dg"]) <= 1e-4 * max(abs(o["dg"]), 1e-3)
    assert g["residual"] == pytest.approx(o["residual"], rel=1e-3)
    assert g["fluid_cells"] == int((cfg["cells"] == 0).sum())
    assert g["steps_done"] == cfg["steps"]


def test_symmetric_tree_mirror_flows_on_gpu(ora):
    cells = I.tree(256, 128, 3, 16, widths=[16, 8, 4, 4], jitter=0)
    assert np.array_equal(cells, cells[::-1])
    lat = L.Lattice(cells, 0.8, 0.03)
    g = lat.solve(1000)
    m = g["m_out"]
    assert len(m) == 8
    assert np.abs(m - m[::-1]).max() <= 1e-5 * np.abs(m).max()


def test_tree_2048_full_size_parity(ora):
    """The 2048 x 1024 four-generation tree at its own parameters, in the
    launch configuration the benchmark uses, for 200 steps."""
    cfg = I.config_tree_2048()
    lat, g, s, o = _run_both(ora, cfg["cells"], cfg["tau"], cfg["u_max"], 200)
    _check_fields(lat, s, cfg["cells"])
    assert abs(g["dp"] - o["dp"]) <= TOL * abs(o["dp"])
    assert g["n_outlets"] == 16
    assert np.abs(g["m_out"] - o["m_out"]).max() <= TOL * np.abs(o["m_out"]).max()


def test_repeat_solves_continue_state(ora):
    cfg = I.config_t_junction()
    lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], residual_every=0)
    for _ in range(3):
        g = lat.solve(100)
    p = ora.make_params(128, 64, cfg["tau"], 1.0, cfg["u_max"])
    s = ora.Solver(p, cfg["cells"], residual_every=0)
    o = s.solve(300)
    assert g["steps_done"] == 300
    assert abs(g["dp"] - o["dp"]) <= TOL * abs(o["dp"])
    _check_fields(lat, s, cfg["cells"])


def test_checkpoint_resume_is_bitwise(ora):
    cfg = I.config_t_junction()
    a = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"])
    a.solve(300)
    saved = a.read(L.FIELD_POPS)
    ga = a.solve(300)
    ua = a.read(L.FIELD_UX)
    b = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"])
    b.load_state(saved)
    gb = b.solve(300)
    assert np.array_equal(ua, b.read(L.FIELD_UX))
    assert ga["dp"] == gb["dp"]


def test_reset_restores_initial_state(ora):
    cfg = I.config_t_junction()
    lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"])
    g1 = lat.solve(200)
    lat.optimize_step(3, 200)
    lat.reset()
    assert np.array_equal(lat.read(L.FIELD_MASK), cfg["cells"])
    g2 = lat.solve(200)
    assert g1["dp"] == g2["dp"] and g2["steps_done"] == 200


def test_argument_errors():
    cfg = I.config_t_junction()
    lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"])
    with pytest.raises(L.LbmError) as e:
        lat.solve(3)
    assert e.value.status == 1
    with pytest.raises(L.LbmError) as e:
        lat.optimize_step(2, 100)  # no field yet
    assert e.value.status == 1
    bad = cfg["cells"].copy()
    bad[0, 5] = 0  # hole in the frame
    with pytest.raises(L.LbmError) as e:
        L.Lattice(bad, 0.8, 0.05)
    assert e.value.status == 2
    with pytest.raises(L.LbmError) as e:
        L.Lattice(I.channel(33, 8), 0.8, 0.05)  # odd nx
    assert e.value.status == 1
    lat.close()


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_reduced_precision_storage_error_reported(ora, prec):
    """16-bit shifted storage: errors against the FP64 oracle are reported; the
    bound here only guards against gross failure (a wrong layout or type)."""
    cfg = I.config_t_junction()
    lat = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], precision=prec)
    g = lat.solve(cfg["steps"])
    p = ora.make_params(128, 64, cfg["tau"], 1.0, cfg["u_max"])
    o = ora.Solver(p, cfg["cells"]).solve(cfg["steps"])
    rel = abs(g["dp"] - o["dp"]) / abs(o["dp"])
    print(f"{prec}: relative dp error {rel:.3e}")
    assert np.isfinite(g["dp"]) and rel < 0.05
